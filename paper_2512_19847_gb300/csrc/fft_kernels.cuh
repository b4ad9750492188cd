// Periodic Helmholtz solve of Algorithm 1, step 2:
//     (D_Delta - kappa_i) theta^(i) = R_i
// by diagonalisation in the discrete Fourier basis (the operator is periodic
// with constant coefficients, so every DFT mode is an eigenvector with
// eigenvalue lam_x(kx) + lam_y(ky) - kappa_i).  Three passes:
//   k_fft_rows_fwd : real row DFTs of R (two rows packed as one complex row),
//                    written as the half spectrum S[y][0..nx/2];
//   k_fft_cols     : per spectral column, DFT along y, division by the
//                    symbol (mode k = 0 set to mean(theta^n), reading G5),
//                    inverse DFT along y, scaled by 1/(nx ny);
//   k_fft_rows_inv : inverse real row DFTs into theta^(i).
// Radix-2 in shared memory: decimation in time from bit-reversed order for
// the forward transforms, decimation in frequency (natural in, bit-reversed
// out) for the inverse ones, so no permutation pass is needed.
#pragma once
#include "common.cuh"

namespace apd {

template <typename T> struct Cplx;
template <> struct Cplx<double> { using type = double2; };
template <> struct Cplx<float> { using type = float2; };

// Twiddles in the transform's own type (no conversion per butterfly).
template <typename T> __device__ __forceinline__ const typename Cplx<T>::type* twiddles(const BatchDev& b);
template <> __device__ __forceinline__ const double2* twiddles<double>(const BatchDev& b) { return b.tw; }
template <> __device__ __forceinline__ const float2* twiddles<float>(const BatchDev& b) { return b.tw32; }

__device__ __forceinline__ int brev(int k, int ln) { return (int)(__brev((unsigned)k) >> (32 - ln)); }

// Complex helpers.  mul_j(z, inv) multiplies by -i (forward) or +i (inverse):
// the twiddle W_{4h}^h of the second stage of a radix-2^2 step.
template <typename C>
__device__ __forceinline__ C cadd(C a, C b) { C r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename C>
__device__ __forceinline__ C csub(C a, C b) { C r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
template <typename C>
__device__ __forceinline__ C cmul_tw(C w, C b, bool inv) {   // w (conjugated when inv) times b
  C r;
  if (inv) { r.x = w.x * b.x + w.y * b.y; r.y = w.x * b.y - w.y * b.x; }
  else { r.x = w.x * b.x - w.y * b.y; r.y = w.x * b.y + w.y * b.x; }
  return r;
}
template <typename C>
__device__ __forceinline__ C mul_j(C a, bool inv) {
  C r;
  if (inv) { r.x = -a.y; r.y = a.x; } else { r.x = a.y; r.y = -a.x; }
  return r;
}

// ntr transforms of length n = 2^ln held back to back in x[], input in
// bit-reversed order, output natural.  Twiddle W_m^p = tw[p * nmax/m].
// Stages are taken two at a time (radix-2^2): each thread loads four
// elements p0 + {0, h, 2h, 3h}, applies stage s (half h, twiddle W_{2h}^pos)
// and stage s+1 (half 2h, twiddles W_{4h}^pos and W_{4h}^pos * W_{4h}^h) in
// registers, and stores them; the first pair of stages has only trivial twiddles.
template <typename T>
__device__ __forceinline__ void fft_dit(typename Cplx<T>::type* x, int ln, int ntr,
                                        const typename Cplx<T>::type* __restrict__ tw, int lnmax,
                                        bool inv, int tid, int nthr) {
  using C = typename Cplx<T>::type;
  const int n = 1 << ln;
  int s = 1;
  for (; s + 1 <= ln; s += 2) {
    const int h = 1 << (s - 1), nq = n >> 2, nb = ntr * nq;
    for (int k = tid; k < nb; k += nthr) {
      const int t = k >> (ln - 2), bi = k & (nq - 1);
      const int pos = bi & (h - 1), grp = bi >> (s - 1);
      const int p0 = t * n + grp * 4 * h + pos;
      C x0 = x[p0], x1 = x[p0 + h], x2 = x[p0 + 2 * h], x3 = x[p0 + 3 * h];
      if (s > 1) {
        const C w1 = tw[pos << (lnmax - s)];
        x1 = cmul_tw(w1, x1, inv);
        x3 = cmul_tw(w1, x3, inv);
      }
      const C a0 = cadd(x0, x1), a1 = csub(x0, x1);
      C a2 = cadd(x2, x3), a3 = csub(x2, x3);
      if (s > 1) {
        const C w2 = tw[pos << (lnmax - s - 1)];
        a2 = cmul_tw(w2, a2, inv);
        a3 = cmul_tw(w2, a3, inv);
      }
      a3 = mul_j(a3, inv);
      x[p0] = cadd(a0, a2);
      x[p0 + 2 * h] = csub(a0, a2);
      x[p0 + h] = cadd(a1, a3);
      x[p0 + 3 * h] = csub(a1, a3);
    }
    __syncthreads();
  }
  if (s == ln) {   // one radix-2 stage left (odd ln)
    const int half = 1 << (s - 1), sh = lnmax - s, nb = ntr * (n >> 1);
    for (int k = tid; k < nb; k += nthr) {
      const int t = k >> (ln - 1), bi = k & ((n >> 1) - 1);
      const int pos = bi & (half - 1), grp = bi >> (s - 1);
      const int i0 = t * n + grp * 2 * half + pos, i1 = i0 + half;
      const C a = x[i0], tb = cmul_tw(tw[pos << sh], x[i1], inv);
      x[i0] = cadd(a, tb);
      x[i1] = csub(a, tb);
    }
    __syncthreads();
  }
}

// Natural-order input, bit-reversed output (decimation in frequency), two
// stages at a time as in fft_dit: stage s (half 2h) then stage s-1 (half h).
template <typename T>
__device__ __forceinline__ void fft_dif(typename Cplx<T>::type* x, int ln, int ntr,
                                        const typename Cplx<T>::type* __restrict__ tw, int lnmax,
                                        bool inv, int tid, int nthr) {
  using C = typename Cplx<T>::type;
  const int n = 1 << ln;
  int s = ln;
  for (; s >= 2; s -= 2) {
    const int h = 1 << (s - 2), nq = n >> 2, nb = ntr * nq;
    for (int k = tid; k < nb; k += nthr) {
      const int t = k >> (ln - 2), bi = k & (nq - 1);
      const int pos = bi & (h - 1), grp = bi >> (s - 2);
      const int p0 = t * n + grp * 4 * h + pos;
      const C x0 = x[p0], x1 = x[p0 + h], x2 = x[p0 + 2 * h], x3 = x[p0 + 3 * h];
      const C b0 = cadd(x0, x2), b1 = cadd(x1, x3);
      C b2 = csub(x0, x2), b3 = csub(x1, x3);
      if (s > 2) {
        const C w2 = tw[pos << (lnmax - s)];
        b2 = cmul_tw(w2, b2, inv);
        b3 = cmul_tw(w2, b3, inv);
      }
      b3 = mul_j(b3, inv);
      C y1 = csub(b0, b1), y3 = csub(b2, b3);
      if (s > 2) {
        const C w1 = tw[pos << (lnmax - s + 1)];
        y1 = cmul_tw(w1, y1, inv);
        y3 = cmul_tw(w1, y3, inv);
      }
      x[p0] = cadd(b0, b1);
      x[p0 + h] = y1;
      x[p0 + 2 * h] = cadd(b2, b3);
      x[p0 + 3 * h] = y3;
    }
    __syncthreads();
  }
  if (s == 1) {   // last radix-2 stage (odd ln): all twiddles are 1
    const int nb = ntr * (n >> 1);
    for (int k = tid; k < nb; k += nthr) {
      const int i0 = 2 * k, i1 = i0 + 1;
      const C a = x[i0], b = x[i1];
      x[i0] = cadd(a, b);
      x[i1] = csub(a, b);
    }
    __syncthreads();
  }
}

template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 8 : 4) k_fft_rows_fwd(const BatchDev* __restrict__ bp) {
  using C = typename Cplx<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* x = reinterpret_cast<C*>(smem_raw);
  const BatchDev& b = *bp;
  const int nitems = b.counts[1], tid = threadIdx.x, nthr = blockDim.x;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int k_inst = find_inst(b.row_start, b.counts[3], it);
    const InstDev& I = b.inst[k_inst];
    const int n = I.nx, ln = I.lnx, ss = I.sstride;
    const int pair0 = (it - b.row_start[k_inst]) * I.row_pairs;
    const int ntr = min(I.row_pairs, (I.ny >> 1) - pair0);
    const T* R = reinterpret_cast<const T*>(I.R);
    for (int e = tid; e < ntr * n; e += nthr) {
      const int p = e >> ln, k = e & (n - 1);
      const size_t row = (size_t)(2 * (pair0 + p));
      C z; z.x = R[row * n + k]; z.y = R[(row + 1) * n + k];
      x[p * n + brev(k, ln)] = z;
    }
    __syncthreads();
    fft_dit<T>(x, ln, ntr, twiddles<T>(b), b.lnmax, false, tid, nthr);
    C* S = reinterpret_cast<C*>(I.S);
    const int nh = (n >> 1) + 1;
    for (int e = tid; e < ntr * nh; e += nthr) {
      const int p = e / nh, k = e - p * nh;
      const C zk = x[p * n + k], zm = x[p * n + ((n - k) & (n - 1))];
      const size_t row = (size_t)(2 * (pair0 + p));
      C A, B;
      A.x = T(0.5) * (zk.x + zm.x); A.y = T(0.5) * (zk.y - zm.y);
      B.x = T(0.5) * (zk.y + zm.y); B.y = T(-0.5) * (zk.x - zm.x);
      S[row * ss + k] = A;
      S[(row + 1) * ss + k] = B;
    }
    __syncthreads();
  }
}

template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 7 : 4) k_fft_cols(const BatchDev* __restrict__ bp, int i) {
  using C = typename Cplx<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* x = reinterpret_cast<C*>(smem_raw);
  __shared__ double red[8];
  __shared__ double s_mean;
  const BatchDev& b = *bp;
  const int nitems = b.counts[2], tid = threadIdx.x, nthr = blockDim.x;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int k_inst = find_inst(b.col_start, b.counts[3], it);
    const InstDev& I = b.inst[k_inst];
    const int n = I.ny, ln = I.lny, ss = I.sstride, nh = (I.nx >> 1) + 1;
    const int col0 = (it - b.col_start[k_inst]) * I.col_group;
    const int ntr = min(I.col_group, nh - col0);
    if (col0 == 0) {
      // mean(theta^n) from the per-tile partial sums, in a fixed order
      const int nt = I.tiles_x * I.tiles_y;
      double acc = 0.0;
      for (int k = tid; k < nt; k += nthr) acc += I.th_part[k];
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
      if ((tid & 31) == 0) red[tid >> 5] = acc;
      __syncthreads();
      if (tid == 0) {
        double sum = 0.0;
        for (int w = 0; w < (nthr + 31) / 32; ++w) sum += red[w];
        s_mean = sum / ((double)I.nx * (double)I.ny);
      }
      __syncthreads();
    }
    C* S = reinterpret_cast<C*>(I.S);
    for (int e = tid; e < ntr * n; e += nthr) {
      const int g = e >> ln, y = e & (n - 1);
      x[g * n + brev(y, ln)] = S[(size_t)y * ss + col0 + g];
    }
    __syncthreads();
    fft_dit<T>(x, ln, ntr, twiddles<T>(b), b.lnmax, false, tid, nthr);
    const double kap = I.kappa[i];
    const double scale = 1.0 / ((double)I.nx * (double)I.ny);
    for (int e = tid; e < ntr * n; e += nthr) {
      const int g = e >> ln, ky = e & (n - 1), kx = col0 + g;
      C v = x[e];
      if (kx == 0 && ky == 0) {
        v.x = T(s_mean); v.y = T(0);
      } else if (sizeof(T) == 8) {
        const double f = scale / (I.lamx[kx] + I.lamy[ky] - kap);
        v.x = T(double(v.x) * f); v.y = T(double(v.y) * f);
      } else {
        const T f = T(scale) / T(I.lamx[kx] + I.lamy[ky] - kap);
        v.x *= f; v.y *= f;
      }
      x[e] = v;
    }
    __syncthreads();
    fft_dif<T>(x, ln, ntr, twiddles<T>(b), b.lnmax, true, tid, nthr);
    for (int e = tid; e < ntr * n; e += nthr) {
      const int g = e >> ln, y = e & (n - 1);
      S[(size_t)y * ss + col0 + g] = x[g * n + brev(y, ln)];
    }
    __syncthreads();
  }
}

template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 8 : 4) k_fft_rows_inv(const BatchDev* __restrict__ bp, int i) {
  using C = typename Cplx<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* x = reinterpret_cast<C*>(smem_raw);
  const BatchDev& b = *bp;
  const int nitems = b.counts[1], tid = threadIdx.x, nthr = blockDim.x;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int k_inst = find_inst(b.row_start, b.counts[3], it);
    const InstDev& I = b.inst[k_inst];
    const int n = I.nx, ln = I.lnx, ss = I.sstride;
    const int pair0 = (it - b.row_start[k_inst]) * I.row_pairs;
    const int ntr = min(I.row_pairs, (I.ny >> 1) - pair0);
    const C* S = reinterpret_cast<const C*>(I.S);
    for (int e = tid; e < ntr * n; e += nthr) {
      const int p = e >> ln, k = e & (n - 1);
      const size_t row = (size_t)(2 * (pair0 + p));
      C A, B;
      if (k <= (n >> 1)) {
        A = S[row * ss + k]; B = S[(row + 1) * ss + k];
      } else {
        A = S[row * ss + (n - k)]; B = S[(row + 1) * ss + (n - k)];
        A.y = -A.y; B.y = -B.y;
      }
      C z; z.x = A.x - B.y; z.y = A.y + B.x;
      x[e] = z;
    }
    __syncthreads();
    fft_dif<T>(x, ln, ntr, twiddles<T>(b), b.lnmax, true, tid, nthr);
    T* th = reinterpret_cast<T*>(I.Xs[i]) + 2 * (size_t)I.nx * I.ny;
    for (int e = tid; e < ntr * n; e += nthr) {
      const int p = e >> ln, m = e & (n - 1);
      const size_t row = (size_t)(2 * (pair0 + p));
      const C z = x[p * n + brev(m, ln)];
      th[row * n + m] = z.x;
      th[(row + 1) * n + m] = z.y;
    }
    __syncthreads();
  }
}

}  // namespace apd
