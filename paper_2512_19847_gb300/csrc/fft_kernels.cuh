// Periodic Helmholtz solve of Algorithm 1, step 2:
//     (D_Delta - kappa_i) theta^(i) = R_i
// by diagonalisation in the discrete Fourier basis (the operator is periodic
// with constant coefficients, so every DFT mode is an eigenvector with
// eigenvalue lam_x(kx) + lam_y(ky) - kappa_i).  Three passes:
//   k_fft_rows_fwd : real row DFTs of R (two rows packed as one complex row),
//                    written as the half spectrum S[y][0..nx/2];
//   k_fft_cols     : per spectral column, DFT along y, division by the
//                    symbol (mode k = 0 set to mean(theta^n): every other term of R has zero mean),
//                    inverse DFT along y, scaled by 1/(nx ny);
//   k_fft_rows_inv : inverse real row DFTs into theta^(i).
// Power-of-two lengths: radix-2^3 passes in shared memory, decimation in time
// from bit-reversed order for the forward transforms, decimation in frequency
// (natural in, bit-reversed out) for the inverse ones, so no permutation pass
// is needed.  Other lengths that factor into 2, 3, 5 and 7: a self-sorting
// mixed-radix transform (below).  Any other length n is transformed by
// Bluestein's chirp-z identity (L. I. Bluestein, 1970): with
// w_m = exp(i pi m^2 / n) and
// jk = (j^2 + k^2 - (k - j)^2) / 2,
//     sum_j x_j exp(-2 pi i jk / n) = conj(w_k) sum_j (x_j conj(w_j)) w_{k-j},
// a circular convolution of length M, the power of two >= 2n - 1, taken with
// two radix-2 transforms of length M and the precomputed DFT of the filter
// (w_m for |m| < n); the inverse transform conjugates chirp and filter.  A
// row or spectral column then occupies M complex values in shared memory.
// Each pass has a power-of-two kernel and a kernel for the other lengths
// (suffix _bs: mixed radix or Bluestein); each takes the work items of its
// kind and skips the others, and a step launches only the kinds its batch
// holds.  When ny is odd, the last row pair
// holds one row (its partner is zero).
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

// Multiplication by the eighth roots W_8^1 = (1 - i)/sqrt2 and W_8^3 = W_8^1 W_8^2
// (conjugated when inv), the constant twiddles inside a radix-2^3 step.
template <typename C>
__device__ __forceinline__ C mul_w8(C a, bool inv) {
  using T = decltype(a.x);
  const T r = T(0.70710678118654752440);
  C b;
  if (inv) { b.x = r * (a.x - a.y); b.y = r * (a.x + a.y); }
  else { b.x = r * (a.x + a.y); b.y = r * (a.y - a.x); }
  return b;
}
template <typename C>
__device__ __forceinline__ C mul_w83(C a, bool inv) { return mul_j(mul_w8(a, inv), inv); }

// Shared-memory index with padding: one spare element after every 2^PS
// elements (PS = 31: none), so that the strided accesses of the butterfly
// passes spread over the 32 banks: with 8-byte (FP32) complex values PS = 4,
// with 16-byte (FP64) values PS = 3, every radix-2^3 pass below reads and
// writes with the minimum number of shared-memory wavefronts.
template <int PS>
__device__ __forceinline__ int pidx(int i) { return PS >= 31 ? i : i + (i >> PS); }
template <typename T>
__host__ __device__ constexpr int pad_shift() { return sizeof(T) == 4 ? 4 : 3; }
// Complex elements a padded region of n values occupies.
__host__ __device__ constexpr int padded_len(int n, int ps) { return ps >= 31 ? n : n + (n >> ps) + 1; }

// ntr transforms of length n = 2^ln held back to back in x[] (element i at
// x[pidx<PS>(i)]), input in bit-reversed order, output natural.  Twiddle
// W_m^p = tw[p * nmax/m].  Stages are taken three at a time (radix-2^3): each
// thread loads eight elements p0 + k h (k = 0..7, h = 2^(s-1)), applies stage s
// (half h, twiddle W_{2h}^pos), stage s+1 (half 2h, W_{4h}^pos and W_{4h}^pos W_4)
// and stage s+2 (half 4h, W_{8h}^pos W_8^k) in registers, and stores them: one
// table twiddle per stage, the rest constant roots.  One or two stages left over
// take a radix-2^2 or radix-2 step; the first step has only constant twiddles.
template <typename T, int PS = 31>
__device__ __forceinline__ void fft_dit(typename Cplx<T>::type* x, int ln, int ntr,
                                        const typename Cplx<T>::type* __restrict__ tw, int lnmax,
                                        bool inv, int tid, int nthr) {
  using C = typename Cplx<T>::type;
  const int n = 1 << ln;
  int s = 1;
  for (; s + 2 <= ln; s += 3) {
    const int h = 1 << (s - 1), ne = n >> 3, nb = ntr * ne;
    for (int k = tid; k < nb; k += nthr) {
      const int t = k >> (ln - 3), bi = k & (ne - 1);
      const int pos = bi & (h - 1), grp = bi >> (s - 1);
      const int q = t * n + grp * 8 * h + pos;
      C v0 = x[pidx<PS>(q)], v1 = x[pidx<PS>(q + h)], v2 = x[pidx<PS>(q + 2 * h)], v3 = x[pidx<PS>(q + 3 * h)];
      C v4 = x[pidx<PS>(q + 4 * h)], v5 = x[pidx<PS>(q + 5 * h)], v6 = x[pidx<PS>(q + 6 * h)], v7 = x[pidx<PS>(q + 7 * h)];
      if (s > 1) {   // stage s: W_{2h}^pos on the odd elements
        const C w1 = tw[pos << (lnmax - s)];
        v1 = cmul_tw(w1, v1, inv); v3 = cmul_tw(w1, v3, inv); v5 = cmul_tw(w1, v5, inv); v7 = cmul_tw(w1, v7, inv);
      }
      C a0 = cadd(v0, v1), a1 = csub(v0, v1), a2 = cadd(v2, v3), a3 = csub(v2, v3);
      C a4 = cadd(v4, v5), a5 = csub(v4, v5), a6 = cadd(v6, v7), a7 = csub(v6, v7);
      if (s > 1) {   // stage s+1: W_{4h}^pos (and W_4 below)
        const C w2 = tw[pos << (lnmax - s - 1)];
        a2 = cmul_tw(w2, a2, inv); a3 = cmul_tw(w2, a3, inv); a6 = cmul_tw(w2, a6, inv); a7 = cmul_tw(w2, a7, inv);
      }
      a3 = mul_j(a3, inv);
      a7 = mul_j(a7, inv);
      C b0 = cadd(a0, a2), b2 = csub(a0, a2), b1 = cadd(a1, a3), b3 = csub(a1, a3);
      C b4 = cadd(a4, a6), b6 = csub(a4, a6), b5 = cadd(a5, a7), b7 = csub(a5, a7);
      if (s > 1) {   // stage s+2: W_{8h}^pos (and W_8^k below)
        const C w3 = tw[pos << (lnmax - s - 2)];
        b4 = cmul_tw(w3, b4, inv); b5 = cmul_tw(w3, b5, inv); b6 = cmul_tw(w3, b6, inv); b7 = cmul_tw(w3, b7, inv);
      }
      b5 = mul_w8(b5, inv);
      b6 = mul_j(b6, inv);
      b7 = mul_w83(b7, inv);
      x[pidx<PS>(q)] = cadd(b0, b4); x[pidx<PS>(q + 4 * h)] = csub(b0, b4);
      x[pidx<PS>(q + h)] = cadd(b1, b5); x[pidx<PS>(q + 5 * h)] = csub(b1, b5);
      x[pidx<PS>(q + 2 * h)] = cadd(b2, b6); x[pidx<PS>(q + 6 * h)] = csub(b2, b6);
      x[pidx<PS>(q + 3 * h)] = cadd(b3, b7); x[pidx<PS>(q + 7 * h)] = csub(b3, b7);
    }
    __syncthreads();
  }
  if (s + 1 == ln) {   // two stages left: radix-2^2
    const int h = 1 << (s - 1), nq = n >> 2, nb = ntr * nq;
    for (int k = tid; k < nb; k += nthr) {
      const int t = k >> (ln - 2), bi = k & (nq - 1);
      const int pos = bi & (h - 1), grp = bi >> (s - 1);
      const int p0 = t * n + grp * 4 * h + pos;
      C x0 = x[pidx<PS>(p0)], x1 = x[pidx<PS>(p0 + h)], x2 = x[pidx<PS>(p0 + 2 * h)], x3 = x[pidx<PS>(p0 + 3 * h)];
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
      x[pidx<PS>(p0)] = cadd(a0, a2);
      x[pidx<PS>(p0 + 2 * h)] = csub(a0, a2);
      x[pidx<PS>(p0 + h)] = cadd(a1, a3);
      x[pidx<PS>(p0 + 3 * h)] = csub(a1, a3);
    }
    __syncthreads();
  } else if (s == ln) {   // one stage left: radix-2
    const int half = 1 << (s - 1), sh = lnmax - s, nb = ntr * (n >> 1);
    for (int k = tid; k < nb; k += nthr) {
      const int t = k >> (ln - 1), bi = k & ((n >> 1) - 1);
      const int pos = bi & (half - 1), grp = bi >> (s - 1);
      const int i0 = t * n + grp * 2 * half + pos, i1 = i0 + half;
      const C a = x[pidx<PS>(i0)], tb = cmul_tw(tw[pos << sh], x[pidx<PS>(i1)], inv);
      x[pidx<PS>(i0)] = cadd(a, tb);
      x[pidx<PS>(i1)] = csub(a, tb);
    }
    __syncthreads();
  }
}

// Natural-order input, bit-reversed output (decimation in frequency), three
// stages at a time as in fft_dit, mirrored: stage s (half 4h, W_{8h}^pos W_8^k
// on the differences), stage s-1 (half 2h, W_{4h}^pos and W_{4h}^pos W_4),
// stage s-2 (half h, W_{2h}^pos), h = 2^(s-3); leftovers as radix-2^2 or radix-2.
template <typename T, int PS = 31>
__device__ __forceinline__ void fft_dif(typename Cplx<T>::type* x, int ln, int ntr,
                                        const typename Cplx<T>::type* __restrict__ tw, int lnmax,
                                        bool inv, int tid, int nthr) {
  using C = typename Cplx<T>::type;
  const int n = 1 << ln;
  int s = ln;
  for (; s >= 3; s -= 3) {
    const int h = 1 << (s - 3), ne = n >> 3, nb = ntr * ne;
    for (int k = tid; k < nb; k += nthr) {
      const int t = k >> (ln - 3), bi = k & (ne - 1);
      const int pos = bi & (h - 1), grp = bi >> (s - 3);
      const int q = t * n + grp * 8 * h + pos;
      const C v0 = x[pidx<PS>(q)], v1 = x[pidx<PS>(q + h)], v2 = x[pidx<PS>(q + 2 * h)], v3 = x[pidx<PS>(q + 3 * h)];
      const C v4 = x[pidx<PS>(q + 4 * h)], v5 = x[pidx<PS>(q + 5 * h)], v6 = x[pidx<PS>(q + 6 * h)], v7 = x[pidx<PS>(q + 7 * h)];
      // stage s: pairs (k, k+4), differences times W_{8h}^pos W_8^k
      C a0 = cadd(v0, v4), a1 = cadd(v1, v5), a2 = cadd(v2, v6), a3 = cadd(v3, v7);
      C a4 = csub(v0, v4), a5 = csub(v1, v5), a6 = csub(v2, v6), a7 = csub(v3, v7);
      a5 = mul_w8(a5, inv);
      a6 = mul_j(a6, inv);
      a7 = mul_w83(a7, inv);
      if (s > 3) {
        const C w3 = tw[pos << (lnmax - s)];
        a4 = cmul_tw(w3, a4, inv); a5 = cmul_tw(w3, a5, inv); a6 = cmul_tw(w3, a6, inv); a7 = cmul_tw(w3, a7, inv);
      }
      // stage s-1: pairs (k, k+2), differences times W_{4h}^pos (W_4 for the odd ones)
      C b0 = cadd(a0, a2), b1 = cadd(a1, a3), b2 = csub(a0, a2), b3 = csub(a1, a3);
      C b4 = cadd(a4, a6), b5 = cadd(a5, a7), b6 = csub(a4, a6), b7 = csub(a5, a7);
      b3 = mul_j(b3, inv);
      b7 = mul_j(b7, inv);
      if (s > 3) {
        const C w2 = tw[pos << (lnmax - s + 1)];
        b2 = cmul_tw(w2, b2, inv); b3 = cmul_tw(w2, b3, inv); b6 = cmul_tw(w2, b6, inv); b7 = cmul_tw(w2, b7, inv);
      }
      // stage s-2: pairs (k, k+1), differences times W_{2h}^pos
      C c1 = csub(b0, b1), c3 = csub(b2, b3), c5 = csub(b4, b5), c7 = csub(b6, b7);
      if (s > 3) {
        const C w1 = tw[pos << (lnmax - s + 2)];
        c1 = cmul_tw(w1, c1, inv); c3 = cmul_tw(w1, c3, inv); c5 = cmul_tw(w1, c5, inv); c7 = cmul_tw(w1, c7, inv);
      }
      x[pidx<PS>(q)] = cadd(b0, b1); x[pidx<PS>(q + h)] = c1;
      x[pidx<PS>(q + 2 * h)] = cadd(b2, b3); x[pidx<PS>(q + 3 * h)] = c3;
      x[pidx<PS>(q + 4 * h)] = cadd(b4, b5); x[pidx<PS>(q + 5 * h)] = c5;
      x[pidx<PS>(q + 6 * h)] = cadd(b6, b7); x[pidx<PS>(q + 7 * h)] = c7;
    }
    __syncthreads();
  }
  if (s == 2) {   // two stages left: radix-2^2 with trivial table twiddles (h = 1)
    const int nq = n >> 2, nb = ntr * nq;
    for (int k = tid; k < nb; k += nthr) {
      const int p0 = 4 * k;
      const C x0 = x[pidx<PS>(p0)], x1 = x[pidx<PS>(p0 + 1)], x2 = x[pidx<PS>(p0 + 2)], x3 = x[pidx<PS>(p0 + 3)];
      const C b0 = cadd(x0, x2), b1 = cadd(x1, x3), b2 = csub(x0, x2);
      const C b3 = mul_j(csub(x1, x3), inv);
      x[pidx<PS>(p0)] = cadd(b0, b1);
      x[pidx<PS>(p0 + 1)] = csub(b0, b1);
      x[pidx<PS>(p0 + 2)] = cadd(b2, b3);
      x[pidx<PS>(p0 + 3)] = csub(b2, b3);
    }
    __syncthreads();
  } else if (s == 1) {   // last radix-2 stage: all twiddles are 1
    const int nb = ntr * (n >> 1);
    for (int k = tid; k < nb; k += nthr) {
      const int i0 = 2 * k, i1 = i0 + 1;
      const C a = x[pidx<PS>(i0)], b = x[pidx<PS>(i1)];
      x[pidx<PS>(i0)] = cadd(a, b);
      x[pidx<PS>(i1)] = csub(a, b);
    }
    __syncthreads();
  }
}

// Circular convolution of ntr sequences of length M = 2^lm held back to back
// in x[] (natural order, zero beyond n) with the Bluestein filter whose DFT is
// filt (bit-reversed order, scaled by 1/M; conjugated when inv): forward
// radix-2 DFT (natural in, bit-reversed out), product with the filter,
// inverse DFT (bit-reversed in, natural out).
template <typename T>
__device__ __forceinline__ void bluestein_conv(typename Cplx<T>::type* x, int lm, int ntr,
                                               const typename Cplx<T>::type* __restrict__ filt,
                                               const typename Cplx<T>::type* __restrict__ tw, int lnmax, bool inv,
                                               int tid, int nthr) {
  fft_dif<T>(x, lm, ntr, tw, lnmax, false, tid, nthr);
  const int m = 1 << lm;
  for (int e = tid; e < ntr * m; e += nthr) x[e] = cmul_tw(filt[e & (m - 1)], x[e], inv);
  __syncthreads();
  fft_dit<T>(x, lm, ntr, tw, lnmax, true, tid, nthr);
}

// mean(theta^n) of instance I from its nt partial sums (one per item of the first
// stage's right-hand side kernel), in a fixed order, into *mean (shared); every thread of the
// block calls it; red holds one value per warp of the block.
__device__ __forceinline__ void theta_mean(const InstDev& I, int nt, double* red, double* mean, int tid, int nthr) {
  // four independent partial sums per thread (their loads in flight together)
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  int k = tid;
  for (; k + 3 * nthr < nt; k += 4 * nthr) {
    a0 += I.th_part[k];
    a1 += I.th_part[k + nthr];
    a2 += I.th_part[k + 2 * nthr];
    a3 += I.th_part[k + 3 * nthr];
  }
  for (; k < nt; k += nthr) a0 += I.th_part[k];
  double acc = (a0 + a1) + (a2 + a3);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((tid & 31) == 0) red[tid >> 5] = acc;
  __syncthreads();
  if (tid == 0) {
    double sum = 0.0;
    for (int w = 0; w < (nthr + 31) / 32; ++w) sum += red[w];
    *mean = sum / ((double)I.nx * (double)I.ny);
  }
  __syncthreads();
}

// ---- power-of-two axes (shared memory padded, pidx<pad_shift<T>()>)

// Threads per block of the power-of-two row passes (FP32 configurable; 1024 / threads
// resident blocks per SM in FP32, three in FP64).
#ifndef APD_ROWS_THREADS32
#define APD_ROWS_THREADS32 256
#endif
template <typename T>
__host__ __device__ constexpr int rows_threads() { return sizeof(T) == 4 ? APD_ROWS_THREADS32 : 256; }
template <typename T>
__host__ __device__ constexpr int rows_min_blocks() { return sizeof(T) == 4 ? 1024 / APD_ROWS_THREADS32 : 3; }

template <typename T>
__global__ void __launch_bounds__(rows_threads<T>(), rows_min_blocks<T>()) k_fft_rows_fwd(const BatchDev* __restrict__ bp) {
  using C = typename Cplx<T>::type;
  constexpr int PS = pad_shift<T>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* x = reinterpret_cast<C*>(smem_raw);
  const BatchDev& b = *bp;
  const int nitems = b.counts[1], tid = threadIdx.x, nthr = blockDim.x;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int k_inst = find_inst(b.row_start, b.counts[3], it);
    const InstDev& I = b.inst[k_inst];
    if (I.chirp[0] || I.mr_npass[0]) continue;      // an item of another length
    const int n = I.nx, ny = I.ny, ln = I.lnx, ss = I.sstride;
    const int pair0 = (it - b.row_start[k_inst]) * I.row_pairs;
    const int ntr = min(I.row_pairs, ((ny + 1) >> 1) - pair0);
    const T* R = reinterpret_cast<const T*>(I.R);
#pragma unroll 4
    for (int e = tid; e < ntr * n; e += nthr) {
      const int p = e >> ln, k = e & (n - 1);
      const size_t row = (size_t)(2 * (pair0 + p));
      C z; z.x = R[row * n + k]; z.y = row + 1 < (size_t)ny ? R[(row + 1) * n + k] : T(0);
      x[pidx<PS>(p * n + brev(k, ln))] = z;
    }
    __syncthreads();
    fft_dit<T, PS>(x, ln, ntr, twiddles<T>(b), b.lnmax, false, tid, nthr);
    C* S = reinterpret_cast<C*>(I.S);
    const int nh = (n >> 1) + 1;
    for (int e = tid; e < ntr * nh; e += nthr) {
      const int p = e / nh, k = e - p * nh;
      const C zk = x[pidx<PS>(p * n + k)], zm = x[pidx<PS>(p * n + ((n - k) & (n - 1)))];
      const size_t row = (size_t)(2 * (pair0 + p));
      C A, B;
      A.x = T(0.5) * (zk.x + zm.x); A.y = T(0.5) * (zk.y - zm.y);
      B.x = T(0.5) * (zk.y + zm.y); B.y = T(-0.5) * (zk.x - zm.x);
      S[row * ss + k] = A;
      if (row + 1 < (size_t)ny) S[(row + 1) * ss + k] = B;
    }
    __syncthreads();
  }
}

// Column pass: a work item is a group of col_group (a power of two) adjacent
// spectral columns, loaded and stored row by row (adjacent threads take
// adjacent columns of one row); the forward transform runs by decimation in
// frequency (natural order in, bit-reversed out) and the inverse by decimation
// in time (bit-reversed in, natural out), so the symbol division takes the
// spectrum in bit-reversed order and no permutation pass is needed.  The FP32
// form runs it with blocks of 512 threads, two per SM (cols_threads<T>; at 2048^2
// its 257 items of four columns then run in one wave: 0.098 ms per step against
// 0.120 with one block of 1024 and 0.143 with 256), the FP64 form with 256 (its
// butterflies keep the FP64 pipe busy either way); the load and store loops are
// unrolled so that several global accesses per thread are in flight.
#ifndef APD_COLS_THREADS32
#define APD_COLS_THREADS32 512
#endif
template <typename T>
__host__ __device__ constexpr int cols_threads() { return sizeof(T) == 4 ? APD_COLS_THREADS32 : 256; }

template <typename T>
__global__ void __launch_bounds__(cols_threads<T>(), sizeof(T) == 4 ? 1024 / APD_COLS_THREADS32 : 2)
    k_fft_cols(const BatchDev* __restrict__ bp, int i) {
  using C = typename Cplx<T>::type;
  constexpr int PS = pad_shift<T>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* x = reinterpret_cast<C*>(smem_raw);
  __shared__ double red[32];
  __shared__ double s_mean;
  const BatchDev& b = *bp;
  const int nitems = b.counts[2], tid = threadIdx.x, nthr = blockDim.x;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int k_inst = find_inst(b.col_start, b.counts[3], it);
    const InstDev& I = b.inst[k_inst];
    if (I.chirp[1] || I.mr_npass[1]) continue;      // an item of another length
    const int n = I.ny, ln = I.lny, ss = I.sstride, nh = (I.nx >> 1) + 1;
    const int G = I.col_group, lg = __ffs(G) - 1;
    const int col0 = (it - b.col_start[k_inst]) * G;
    const int ntr = min(G, nh - col0);
    if (col0 == 0) theta_mean(I, b.rhs_start[k_inst + 1] - b.rhs_start[k_inst], red, &s_mean, tid, nthr);
    C* S = reinterpret_cast<C*>(I.S);
#pragma unroll 4
    for (int e = tid; e < (n << lg); e += nthr) {
      const int y = e >> lg, g = e & (G - 1);
      if (g < ntr) x[pidx<PS>(g * n + y)] = S[(size_t)y * ss + col0 + g];
    }
    __syncthreads();
    fft_dif<T, PS>(x, ln, ntr, twiddles<T>(b), b.lnmax, false, tid, nthr);
    const double kap = I.kappa[i];
    const double scale = 1.0 / ((double)I.nx * (double)I.ny);
    for (int e = tid; e < ntr * n; e += nthr) {
      const int g = e >> ln, ky = brev(e & (n - 1), ln), kx = col0 + g;
      C v = x[pidx<PS>(e)];
      if (kx == 0 && ky == 0) {
        v.x = T(s_mean); v.y = T(0);
      } else if (sizeof(T) == 8) {
        const double f = scale * rcp_newton(I.lamx[kx] + I.lamy[ky] - kap);
        v.x = T(double(v.x) * f); v.y = T(double(v.y) * f);
      } else {
        // FP32 form: the symbol in FP32 from the tables rounded once on the host
        const float f = I.hscale32 * __frcp_rn(I.lamx32[kx] + I.lamy32[ky] - I.k32.kappa[i]);
        v.x *= T(f); v.y *= T(f);
      }
      x[pidx<PS>(e)] = v;
    }
    __syncthreads();
    fft_dit<T, PS>(x, ln, ntr, twiddles<T>(b), b.lnmax, true, tid, nthr);
#pragma unroll 4
    for (int e = tid; e < (n << lg); e += nthr) {
      const int y = e >> lg, g = e & (G - 1);
      if (g < ntr) S[(size_t)y * ss + col0 + g] = x[pidx<PS>(g * n + y)];
    }
    __syncthreads();
  }
}

template <typename T>
__global__ void __launch_bounds__(rows_threads<T>(), rows_min_blocks<T>()) k_fft_rows_inv(const BatchDev* __restrict__ bp, int i) {
  using C = typename Cplx<T>::type;
  constexpr int PS = pad_shift<T>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* x = reinterpret_cast<C*>(smem_raw);
  const BatchDev& b = *bp;
  const int nitems = b.counts[1], tid = threadIdx.x, nthr = blockDim.x;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int k_inst = find_inst(b.row_start, b.counts[3], it);
    const InstDev& I = b.inst[k_inst];
    if (I.chirp[0] || I.mr_npass[0]) continue;      // an item of another length
    const int n = I.nx, ny = I.ny, ln = I.lnx, ss = I.sstride;
    const int pair0 = (it - b.row_start[k_inst]) * I.row_pairs;
    const int ntr = min(I.row_pairs, ((ny + 1) >> 1) - pair0);
    const C* S = reinterpret_cast<const C*>(I.S);
#pragma unroll 4
    for (int e = tid; e < ntr * n; e += nthr) {
      const int p = e >> ln, k = e & (n - 1);
      const size_t row = (size_t)(2 * (pair0 + p));
      const bool two = row + 1 < (size_t)ny;
      C A, B;
      B.x = B.y = T(0);
      if (k <= (n >> 1)) {
        A = S[row * ss + k];
        if (two) B = S[(row + 1) * ss + k];
      } else {
        A = S[row * ss + (n - k)];
        if (two) B = S[(row + 1) * ss + (n - k)];
        A.y = -A.y; B.y = -B.y;
      }
      C z; z.x = A.x - B.y; z.y = A.y + B.x;
      x[pidx<PS>(e)] = z;
    }
    __syncthreads();
    fft_dif<T, PS>(x, ln, ntr, twiddles<T>(b), b.lnmax, true, tid, nthr);
    T* th = reinterpret_cast<T*>(I.Xs[i]) + 2 * (size_t)I.nx * I.ny;
    for (int e = tid; e < ntr * n; e += nthr) {
      const int p = e >> ln, m = e & (n - 1);
      const size_t row = (size_t)(2 * (pair0 + p));
      const C z = x[pidx<PS>(p * n + brev(m, ln))];
      th[row * n + m] = z.x;
      if (row + 1 < (size_t)ny) th[(row + 1) * n + m] = z.y;
    }
    __syncthreads();
  }
}

// ---- mixed radix: lengths 2^a 3^b 5^c 7^d that are not powers of two, by
// Stockham's self-sorting formulation (natural order in and out, ping-pong
// between two buffers of n values).  With Ns the product of the radices of
// the passes before, a pass of radix R takes, for each j < n/R with k = j mod Ns,
// the R values src[j + r n/R] times W_{Ns R}^{k r}, transforms them with an
// R-point DFT and writes them to dst[(j - k) R + k + r Ns].

// cos and sin of 2 pi q / R, q = 1 .. (R-1)/2, for the odd radices.
__device__ __forceinline__ constexpr double root_cos(int R, int q) {
  return R == 3 ? -0.5
       : R == 5 ? (q == 1 ? 0.3090169943749474241022934 : -0.8090169943749474241022934)
       : (q == 1 ? 0.6234898018587335305250049 : q == 2 ? -0.2225209339563144042889026 : -0.9009688679024191262361023);
}
__device__ __forceinline__ constexpr double root_sin(int R, int q) {
  return R == 3 ? 0.8660254037844386467637232
       : R == 5 ? (q == 1 ? 0.9510565162951535721164393 : 0.5877852522924731291687060)
       : (q == 1 ? 0.7818314824680298087084445 : q == 2 ? 0.9749279121818236070181317 : 0.4338837391175581204757683);
}

// R-point DFT of v in place (exp(-2 pi i ab/R); conjugate roots when inv).  Odd R:
// opposite inputs are paired, y_a = v_0 + sum_b [(v_b + v_{R-b}) cos - i (v_b - v_{R-b}) sin](2 pi ab/R).
template <int R, typename C>
__device__ __forceinline__ void small_dft(C* v, bool inv) {
  using T = decltype(v[0].x);
  if constexpr (R == 2) {
    const C a = v[0];
    v[0] = cadd(a, v[1]);
    v[1] = csub(a, v[1]);
  } else if constexpr (R == 4) {
    const C t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]), t2 = cadd(v[1], v[3]), t3 = mul_j(csub(v[1], v[3]), inv);
    v[0] = cadd(t0, t2);
    v[2] = csub(t0, t2);
    v[1] = cadd(t1, t3);
    v[3] = csub(t1, t3);
  } else {
    constexpr int H = (R - 1) / 2;
    C sp[H], dm[H], out[R];
    C y0 = v[0];
#pragma unroll
    for (int b = 1; b <= H; ++b) {
      sp[b - 1] = cadd(v[b], v[R - b]);
      dm[b - 1] = csub(v[b], v[R - b]);
      y0 = cadd(y0, sp[b - 1]);
    }
    out[0] = y0;
#pragma unroll
    for (int a = 1; a <= H; ++a) {
      C re = v[0], im;
      im.x = T(0); im.y = T(0);
#pragma unroll
      for (int b = 1; b <= H; ++b) {
        const int q = (a * b) % R, qq = q <= H ? q : R - q;
        const T c = T(root_cos(R, qq)), sn = q <= H ? T(root_sin(R, qq)) : -T(root_sin(R, qq));
        re.x += c * sp[b - 1].x; re.y += c * sp[b - 1].y;
        im.x += sn * dm[b - 1].x; im.y += sn * dm[b - 1].y;
      }
      C ya, yb;   // re -+ i im (forward), re +- i im (inverse)
      if (!inv) { ya.x = re.x + im.y; ya.y = re.y - im.x; yb.x = re.x - im.y; yb.y = re.y + im.x; }
      else { ya.x = re.x - im.y; ya.y = re.y + im.x; yb.x = re.x + im.y; yb.y = re.y - im.x; }
      out[a] = ya;
      out[R - a] = yb;
    }
#pragma unroll
    for (int a = 0; a < R; ++a) v[a] = out[a];
  }
}

template <typename T, int R>
__device__ __forceinline__ void stockham_pass(typename Cplx<T>::type* x, int m, int n, int ntr, int Ns, int src_off,
                                              const typename Cplx<T>::type* __restrict__ tw, bool inv, int tid,
                                              int nthr) {
  using C = typename Cplx<T>::type;
  const int nr = n / R, dst_off = n - src_off, tws = n / (Ns * R);
  for (int e = tid; e < ntr * nr; e += nthr) {
    const int p = e / nr, j = e - p * nr, k = j % Ns;
    const C* src = x + p * m + src_off;
    C* dst = x + p * m + dst_off;
    C v[R];
    v[0] = src[j];
#pragma unroll
    for (int r = 1; r < R; ++r) v[r] = cmul_tw(tw[k * r * tws], src[j + r * nr], inv);
    small_dft<R>(v, inv);
    const int d0 = (j - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) dst[d0 + r * Ns] = v[r];
  }
  __syncthreads();
}

// ntr transforms of length n (plan: npass radices, 4 bits each, first pass in the
// low bits), transform p in x + p m, starting in the buffer at offset off (0 or n);
// returns the offset of the buffer that holds the result.  tw[q] = W_n^q, q < n.
template <typename T>
__device__ __forceinline__ int stockham(typename Cplx<T>::type* x, int m, int n, int ntr, unsigned plan, int npass,
                                        const typename Cplx<T>::type* __restrict__ tw, bool inv, int off, int tid,
                                        int nthr) {
  int Ns = 1;
  for (int q = 0; q < npass; ++q) {
    const int R = (int)((plan >> (4 * q)) & 15u);
    if (R == 4) stockham_pass<T, 4>(x, m, n, ntr, Ns, off, tw, inv, tid, nthr);
    else if (R == 2) stockham_pass<T, 2>(x, m, n, ntr, Ns, off, tw, inv, tid, nthr);
    else if (R == 3) stockham_pass<T, 3>(x, m, n, ntr, Ns, off, tw, inv, tid, nthr);
    else if (R == 5) stockham_pass<T, 5>(x, m, n, ntr, Ns, off, tw, inv, tid, nthr);
    else stockham_pass<T, 7>(x, m, n, ntr, Ns, off, tw, inv, tid, nthr);
    off = n - off;
    Ns *= R;
  }
  return off;
}

// ---- axes whose length is not a power of two: mixed radix where the length
// factors into 2, 3, 5 and 7, else Bluestein; x holds ntr regions of m = 2^ln
// values (the Bluestein convolution length, >= 2n: room for the two mixed-radix
// buffers as well) back to back

template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 3) k_fft_rows_fwd_bs(const BatchDev* __restrict__ bp) {
  using C = typename Cplx<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* x = reinterpret_cast<C*>(smem_raw);
  const BatchDev& b = *bp;
  const int nitems = b.counts[1], tid = threadIdx.x, nthr = blockDim.x;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int k_inst = find_inst(b.row_start, b.counts[3], it);
    const InstDev& I = b.inst[k_inst];
    const C* ch = reinterpret_cast<const C*>(I.chirp[0]);
    if (!ch && !I.mr_npass[0]) continue;            // a power-of-two item
    const int n = I.nx, ny = I.ny, ln = I.lnx, m = 1 << ln, ss = I.sstride;
    const int pair0 = (it - b.row_start[k_inst]) * I.row_pairs;
    const int ntr = min(I.row_pairs, ((ny + 1) >> 1) - pair0);
    const T* R = reinterpret_cast<const T*>(I.R);
    if (I.mr_npass[0]) {
      for (int e = tid; e < ntr * n; e += nthr) {
        const int p = e / n, k = e - p * n;
        const size_t row = (size_t)(2 * (pair0 + p));
        C z;
        z.x = R[row * n + k];
        z.y = row + 1 < (size_t)ny ? R[(row + 1) * n + k] : T(0);
        x[p * m + k] = z;
      }
      __syncthreads();
      const int off = stockham<T>(x, m, n, ntr, I.mr_plan[0], I.mr_npass[0], reinterpret_cast<const C*>(I.mr_tw[0]),
                                  false, 0, tid, nthr);
      C* S = reinterpret_cast<C*>(I.S);
      const int nh = (n >> 1) + 1;
      for (int e = tid; e < ntr * nh; e += nthr) {
        const int p = e / nh, k = e - p * nh, km = k == 0 ? 0 : n - k;
        const C zk = x[p * m + off + k], zm = x[p * m + off + km];
        const size_t row = (size_t)(2 * (pair0 + p));
        C A, B;
        A.x = T(0.5) * (zk.x + zm.x); A.y = T(0.5) * (zk.y - zm.y);
        B.x = T(0.5) * (zk.y + zm.y); B.y = T(-0.5) * (zk.x - zm.x);
        S[row * ss + k] = A;
        if (row + 1 < (size_t)ny) S[(row + 1) * ss + k] = B;
      }
      __syncthreads();
      continue;
    }
    for (int e = tid; e < ntr * m; e += nthr) {
      const int p = e >> ln, k = e & (m - 1);
      const size_t row = (size_t)(2 * (pair0 + p));
      C z;
      z.x = T(0); z.y = T(0);
      if (k < n) {
        z.x = R[row * n + k];
        if (row + 1 < (size_t)ny) z.y = R[(row + 1) * n + k];
        z = cmul_tw(ch[k], z, false);
      }
      x[e] = z;
    }
    __syncthreads();
    bluestein_conv<T>(x, ln, ntr, reinterpret_cast<const C*>(I.filt[0]), twiddles<T>(b), b.lnmax, false, tid, nthr);
    C* S = reinterpret_cast<C*>(I.S);
    const int nh = (n >> 1) + 1;
    for (int e = tid; e < ntr * nh; e += nthr) {
      const int p = e / nh, k = e - p * nh, km = k == 0 ? 0 : n - k;
      const C zk = cmul_tw(ch[k], x[p * m + k], false), zm = cmul_tw(ch[km], x[p * m + km], false);
      const size_t row = (size_t)(2 * (pair0 + p));
      C A, B;
      A.x = T(0.5) * (zk.x + zm.x); A.y = T(0.5) * (zk.y - zm.y);
      B.x = T(0.5) * (zk.y + zm.y); B.y = T(-0.5) * (zk.x - zm.x);
      S[row * ss + k] = A;
      if (row + 1 < (size_t)ny) S[(row + 1) * ss + k] = B;
    }
    __syncthreads();
  }
}

// The forward Bluestein convolution differs from the spectrum along y by the
// factor conj(w_ky), which the inverse transform's input chirp w_ky cancels,
// so the division by the symbol applies to the convolution directly.
template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 3) k_fft_cols_bs(const BatchDev* __restrict__ bp, int i) {
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
    const C* ch = reinterpret_cast<const C*>(I.chirp[1]);
    if (!ch && !I.mr_npass[1]) continue;            // a power-of-two item
    const C* filt = reinterpret_cast<const C*>(I.filt[1]);
    const int n = I.ny, ln = I.lny, m = 1 << ln, ss = I.sstride, nh = (I.nx >> 1) + 1;
    const int col0 = (it - b.col_start[k_inst]) * I.col_group;
    const int ntr = min(I.col_group, nh - col0);
    if (col0 == 0) theta_mean(I, b.rhs_start[k_inst + 1] - b.rhs_start[k_inst], red, &s_mean, tid, nthr);
    C* S = reinterpret_cast<C*>(I.S);
    if (I.mr_npass[1]) {
      const C* tw = reinterpret_cast<const C*>(I.mr_tw[1]);
      for (int e = tid; e < ntr * n; e += nthr) {
        const int g = e / n, y = e - g * n;
        x[g * m + y] = S[(size_t)y * ss + col0 + g];
      }
      __syncthreads();
      const int off = stockham<T>(x, m, n, ntr, I.mr_plan[1], I.mr_npass[1], tw, false, 0, tid, nthr);
      const double kap = I.kappa[i];
      const double scale = 1.0 / ((double)I.nx * (double)I.ny);
      for (int e = tid; e < ntr * n; e += nthr) {
        const int g = e / n, ky = e - g * n, kx = col0 + g;
        C v = x[g * m + off + ky];
        if (kx == 0 && ky == 0) {
          v.x = T(s_mean); v.y = T(0);
        } else {
          const double f = scale * rcp_newton(I.lamx[kx] + I.lamy[ky] - kap);
          v.x = T(double(v.x) * f); v.y = T(double(v.y) * f);
        }
        x[g * m + off + ky] = v;
      }
      __syncthreads();
      const int off2 = stockham<T>(x, m, n, ntr, I.mr_plan[1], I.mr_npass[1], tw, true, off, tid, nthr);
      for (int e = tid; e < ntr * n; e += nthr) {
        const int g = e / n, y = e - g * n;
        S[(size_t)y * ss + col0 + g] = x[g * m + off2 + y];
      }
      __syncthreads();
      continue;
    }
    for (int e = tid; e < ntr * m; e += nthr) {
      const int g = e >> ln, y = e & (m - 1);
      C z;
      z.x = T(0); z.y = T(0);
      if (y < n) z = cmul_tw(ch[y], S[(size_t)y * ss + col0 + g], false);
      x[e] = z;
    }
    __syncthreads();
    bluestein_conv<T>(x, ln, ntr, filt, twiddles<T>(b), b.lnmax, false, tid, nthr);
    const double kap = I.kappa[i];
    const double scale = 1.0 / ((double)I.nx * (double)I.ny);
    for (int e = tid; e < ntr * m; e += nthr) {
      const int g = e >> ln, ky = e & (m - 1), kx = col0 + g;
      C v = x[e];
      if (ky >= n) {
        v.x = T(0); v.y = T(0);
      } else if (kx == 0 && ky == 0) {
        v.x = T(s_mean); v.y = T(0);
      } else {
        const double f = scale * rcp_newton(I.lamx[kx] + I.lamy[ky] - kap);
        v.x = T(double(v.x) * f); v.y = T(double(v.y) * f);
      }
      x[e] = v;
    }
    __syncthreads();
    bluestein_conv<T>(x, ln, ntr, filt, twiddles<T>(b), b.lnmax, true, tid, nthr);
    for (int e = tid; e < ntr * m; e += nthr) {
      const int g = e >> ln, y = e & (m - 1);
      if (y < n) S[(size_t)y * ss + col0 + g] = cmul_tw(ch[y], x[e], true);
    }
    __syncthreads();
  }
}

template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 4 : 3) k_fft_rows_inv_bs(const BatchDev* __restrict__ bp, int i) {
  using C = typename Cplx<T>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* x = reinterpret_cast<C*>(smem_raw);
  const BatchDev& b = *bp;
  const int nitems = b.counts[1], tid = threadIdx.x, nthr = blockDim.x;
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int k_inst = find_inst(b.row_start, b.counts[3], it);
    const InstDev& I = b.inst[k_inst];
    const C* ch = reinterpret_cast<const C*>(I.chirp[0]);
    if (!ch && !I.mr_npass[0]) continue;            // a power-of-two item
    const int n = I.nx, ny = I.ny, ln = I.lnx, m = 1 << ln, ss = I.sstride;
    const int pair0 = (it - b.row_start[k_inst]) * I.row_pairs;
    const int ntr = min(I.row_pairs, ((ny + 1) >> 1) - pair0);
    const C* S = reinterpret_cast<const C*>(I.S);
    if (I.mr_npass[0]) {
      for (int e = tid; e < ntr * n; e += nthr) {
        const int p = e / n, k = e - p * n;
        const size_t row = (size_t)(2 * (pair0 + p));
        const bool two = row + 1 < (size_t)ny;
        const int kk = k <= (n >> 1) ? k : n - k;   // Hermitian symmetry of a real row
        C A = S[row * ss + kk], B;
        B.x = B.y = T(0);
        if (two) B = S[(row + 1) * ss + kk];
        if (kk != k) { A.y = -A.y; B.y = -B.y; }
        C z;
        z.x = A.x - B.y; z.y = A.y + B.x;
        x[p * m + k] = z;
      }
      __syncthreads();
      const int off = stockham<T>(x, m, n, ntr, I.mr_plan[0], I.mr_npass[0], reinterpret_cast<const C*>(I.mr_tw[0]),
                                  true, 0, tid, nthr);
      T* th = reinterpret_cast<T*>(I.Xs[i]) + 2 * (size_t)I.nx * I.ny;
      for (int e = tid; e < ntr * n; e += nthr) {
        const int p = e / n, mm = e - p * n;
        const size_t row = (size_t)(2 * (pair0 + p));
        const C z = x[p * m + off + mm];
        th[row * n + mm] = z.x;
        if (row + 1 < (size_t)ny) th[(row + 1) * n + mm] = z.y;
      }
      __syncthreads();
      continue;
    }
    for (int e = tid; e < ntr * m; e += nthr) {
      const int p = e >> ln, k = e & (m - 1);
      const size_t row = (size_t)(2 * (pair0 + p));
      const bool two = row + 1 < (size_t)ny;
      C A, B, z;
      A.x = A.y = B.x = B.y = z.x = z.y = T(0);
      if (k < n) {
        const int kk = k <= (n >> 1) ? k : n - k;   // Hermitian symmetry of a real row
        A = S[row * ss + kk];
        if (two) B = S[(row + 1) * ss + kk];
        if (kk != k) { A.y = -A.y; B.y = -B.y; }
        z.x = A.x - B.y; z.y = A.y + B.x;
        z = cmul_tw(ch[k], z, true);
      }
      x[e] = z;
    }
    __syncthreads();
    bluestein_conv<T>(x, ln, ntr, reinterpret_cast<const C*>(I.filt[0]), twiddles<T>(b), b.lnmax, true, tid, nthr);
    T* th = reinterpret_cast<T*>(I.Xs[i]) + 2 * (size_t)I.nx * I.ny;
    for (int e = tid; e < ntr * m; e += nthr) {
      const int p = e >> ln, mm = e & (m - 1);
      if (mm >= n) continue;
      const size_t row = (size_t)(2 * (pair0 + p));
      const C z = cmul_tw(ch[mm], x[e], true);
      th[row * n + mm] = z.x;
      if (row + 1 < (size_t)ny) th[(row + 1) * n + mm] = z.y;
    }
    __syncthreads();
  }
}

}  // namespace apd
