// Tile kernels of one IMEX stage (Algorithm 1 with the operators of Sec. 3.2).
//
//   k_explicit(j): explicit term of step 1 for stage j,
//       E^(j) = (tau/4) D0_LF . B(u^(j)) + tau eps^2 D_LF q^(j) - F(u^(j)),
//     the derived operators of stage j that later stages reuse
//       D_0 . u^(j), D_Delta theta^(j), D_LF . B(v^(j)) (partner u^(j)) + D_0 theta^(j),
//     and step 1 of stage j+1: the closed-form v^(j+1), once per cell.
//   k_rhs(i):  the right-hand side R_i of the Helmholtz equation (step 2), by rows.
//   k_update(i): step 3 (u^(i)) and step 4 (closed-form q^(i)); for the last stage
//     with close_step set, also the close of the step (GSA: X^{n+1} = X^(s); the
//     FP32 forms pack the populations and sum the next step's moments), written
//     to the other buffer of the double-buffered state.
//
// Every kernel is a persistent loop over the batch's tile list.  The halo'd
// plane tiles a kernel reads are staged into shared memory by TMA (one bulk
// tensor copy per plane, completing on an mbarrier), double-buffered so that
// the copies of the next tile run while the current one is computed.
// Upwind fluxes are then computed one axis at a time: for every flux/partner
// pair the Lax-Friedrichs splitting g+- = (g +- U)/2 and the curvature part
// of the WENO5 smoothness indicators are evaluated once per point, then each
// interface flux once, then differenced.  The WENO fluxes take the split without
// its factor 1/2 (g +- U, with eps_W scaled by 4): every operation of a WENO
// reconstruction is homogeneous under a power-of-two scaling of its inputs once
// eps_W scales with the indicators, so the interface flux comes out exactly twice
// the one of (g +- U)/2, and the 1/2 joins 1/dx in the flux difference (flux_scale).
#pragma once
#include <type_traits>
#include "common.cuh"
#include "io_kernels.cuh"
#include "tma.cuh"

namespace apd {

enum NeedBits { NEED_E = 1, NEED_DU = 2, NEED_LTH = 4, NEED_DLFB = 16, NEED_V = 32 };

// Geometry of a staged plane tile: rows y0-H .. y0+TY+H-1, columns
// x0-4 .. x0+TX+3 (row stride BW); logical tile column 0 (x = x0-H) sits at
// shared-memory column XO.
template <typename T, int SCHEME, int TX, int TY>
struct Geo {
  static constexpr int H = halo_of(SCHEME), CH = central_halo(SCHEME);
  static constexpr int W = TX + 2 * H, HH = TY + 2 * H;
  static constexpr int BW = TX + 8, BH = HH;
  static constexpr int XO = 4 - H;
  static constexpr int PL = ((BW * BH * (int)sizeof(T) + 127) / 128) * 128 / (int)sizeof(T);
  static constexpr unsigned PLANE_BYTES = (unsigned)(BW * BH * sizeof(T));
  static constexpr int C00 = H * BW + 4;                // interior cell (0, 0)
  static constexpr int NX = TY * (TX + 1), NY = (TY + 1) * TX;
  static constexpr int LS = (TY * W > HH * TX) ? TY * W : HH * TX;
  // FP32 WENO5 computes its fluxes in register runs: no split scratch, no partner planes
  static constexpr bool RUNS = SCHEME == WENO5_C4 && sizeof(T) == 4;
  // FP64 WENO5 update: the passes of both axes run together (split scratch for both
  // axes at once), its planes staged single-buffered to leave room for it
  static constexpr bool MERGED = SCHEME == WENO5_C4 && sizeof(T) == 8;
  static constexpr int NBUF_U = MERGED ? 1 : 2;               // staged plane buffers of k_update
  static constexpr int LSX = TY * W, LSY = HH * TX;           // split points per pair, x and y
  static constexpr int SPLIT_PER_PAIR = (SCHEME == LF1_C2 || RUNS) ? 0 : 4 * LS;
  static constexpr int SPLIT_U_PER_PAIR = (SCHEME == LF1_C2 || RUNS) ? 0 : (MERGED ? 4 * (LSX + LSY) : 4 * LS);
  // shared memory besides the staged planes, and its element count
  static constexpr int EXPLICIT_EXTRA = 3 * SPLIT_PER_PAIR + 3 * NX + 3 * NY;
  static constexpr int UPDATE_EXTRA = (RUNS ? 0 : 2 * PL) + 2 * SPLIT_U_PER_PAIR + 2 * NX + 2 * NY;
};

// The planes a kernel stages, packed 6 bits each (buffer << 3 | plane) so the
// list stays in registers.  Buffer j: the stage values X^(j) (X^(1) = X^n for CK/ARS tableaux).
struct PlaneList {
  uint64_t bits = 0;
  int n = 0;
  __device__ __forceinline__ void add(int buf, int plane) { bits |= uint64_t((buf << 3) | plane) << (6 * n); ++n; }
  __device__ __forceinline__ int buf(int k) const { return int(bits >> (6 * k + 3)) & 7; }
  __device__ __forceinline__ int plane(int k) const { return int(bits >> (6 * k)) & 7; }
};

__device__ __forceinline__ const void* stage_buffer(const InstDev& I, int buf) { return I.Xs[buf]; }
__device__ __forceinline__ const void* stage_map(const InstDev& I, int buf) {
  return reinterpret_cast<const char*>(I.tmap) + 128 * buf;
}

struct TileRef { int inst, tile, x0, y0; };

template <int TX, int TY>
__device__ __forceinline__ TileRef decode_tile(const BatchDev& b, int it) {
  TileRef t;
  t.inst = find_inst(b.tile_start, b.counts[3], it);
  const InstDev& I = b.inst[t.inst];
  t.tile = it - b.tile_start[t.inst];
  const int tyi = t.tile / I.tiles_x;
  t.x0 = (t.tile - tyi * I.tiles_x) * TX;
  t.y0 = tyi * TY;
  return t;
}

// Plain loads of the staged box with periodic wrap (instances without TMA staging).
// A ragged tile at the high edge of the grid stages periodic images past the last
// cell as well: its cells beyond the grid are computed but not stored.
template <typename T, class G>
__device__ __forceinline__ void stage_plain(const InstDev& I, const PlaneList& pr, T* dst, int x0, int y0, int tid,
                                            int nthr) {
  const int nx = I.nx, ny = I.ny;
  const size_t pl = (size_t)nx * ny;
  for (int k = 0; k < pr.n; ++k) {
    const T* g = reinterpret_cast<const T*>(stage_buffer(I, pr.buf(k))) + (size_t)pr.plane(k) * pl;
    for (int e = tid; e < G::BW * G::BH; e += nthr) {
      const int r = e / G::BW, c = e - r * G::BW;
      const int gx = x0 - 4 + c, gy = y0 - G::H + r;
      dst[k * G::PL + e] = g[(size_t)wrap_index(gy, ny) * nx + wrap_index(gx, nx)];
    }
  }
}

// After a TMA copy of a box that crosses the grid edge: write the periodic images into
// the box cells outside the grid (which the copy filled with zero), visiting only those
// cells (the rows above and below the grid, then the columns left and right of it on the
// other rows), every staged plane's value of one cell loaded before any is stored.
template <typename T, class G>
__device__ __forceinline__ void stage_edges(const InstDev& I, const PlaneList& pr, T* dst, int x0, int y0, int tid,
                                            int nthr) {
  constexpr int MAXP = 3 + 2 * (APD_MAXS - 1);   // the most planes a kernel stages
  const int nx = I.nx, ny = I.ny;
  const size_t pl = (size_t)nx * ny;
  const int bx0 = x0 - 4, by0 = y0 - G::H;
  const int rlo = max(0, -by0), rhi = max(0, by0 + G::BH - ny);
  const int clo = max(0, -bx0), chi = max(0, bx0 + G::BW - nx);
  const int nfull = (rlo + rhi) * G::BW, ncol = clo + chi;
  const int total = nfull + (G::BH - rlo - rhi) * ncol;
  const T* src[MAXP];
#pragma unroll
  for (int k = 0; k < MAXP; ++k)
    src[k] = k < pr.n ? reinterpret_cast<const T*>(stage_buffer(I, pr.buf(k))) + (size_t)pr.plane(k) * pl : nullptr;
  for (int e = tid; e < total; e += nthr) {
    int r, c;
    if (e < nfull) {
      const int q = e / G::BW;
      c = e - q * G::BW;
      r = q < rlo ? q : G::BH - rhi + (q - rlo);
    } else {
      const int e2 = e - nfull, q = e2 / ncol, w = e2 - q * ncol;
      r = rlo + q;
      c = w < clo ? w : G::BW - chi + (w - clo);
    }
    const size_t go = (size_t)wrap_index(by0 + r, ny) * nx + wrap_index(bx0 + c, nx);
    const int so = r * G::BW + c;
    T v[MAXP];
#pragma unroll
    for (int k = 0; k < MAXP; ++k)
      if (k < pr.n) v[k] = src[k][go];
#pragma unroll
    for (int k = 0; k < MAXP; ++k)
      if (k < pr.n) dst[k * G::PL + so] = v[k];
  }
}

template <class G>
__device__ __forceinline__ bool tile_on_edge(const InstDev& I, int x0, int y0) {
  return x0 - 4 < 0 || x0 - 4 + G::BW > I.nx || y0 - G::H < 0 || y0 - G::H + G::BH > I.ny;
}

// Start staging tile `it` into dst: TMA copies issued by thread 0, or plain loads by all threads.
template <typename T, class G, int TX, int TY>
__device__ __forceinline__ void stage_begin(const BatchDev& b, int it, const PlaneList& pr, T* dst, uint64_t* bar,
                                            int tid, int nthr) {
  const TileRef t = decode_tile<TX, TY>(b, it);
  const InstDev& I = b.inst[t.inst];
  if (I.tma) {
    if (tid == 0) {
      fence_proxy_async();
      mbar_arrive_expect_tx(bar, (unsigned)pr.n * G::PLANE_BYTES);
      for (int k = 0; k < pr.n; ++k)
        tma_load_3d(dst + k * G::PL, stage_map(I, pr.buf(k)), t.x0 - 4, t.y0 - G::H, pr.plane(k), bar);
    }
  } else {
    stage_plain<T, G>(I, pr, dst, t.x0, t.y0, tid, nthr);
  }
}

// The persistent, double-buffered tile loop: body(I, tile, staged planes) runs
// for every tile of the batch assigned to this block.
template <typename T, class G, int TX, int TY, int NB = 2, class Body>
__device__ __forceinline__ void tile_loop(const BatchDev& b, const PlaneList& pr, T* stage0, uint64_t* bars, int tid,
                                          Body&& body) {
  constexpr int NT = TX * TY;
  const int ntiles = b.counts[0];
  const int bstride = pr.n * G::PL;       // buffer 1 starts at stage0 + bstride
  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  unsigned phase = 0u;                    // bit c: parity of the next phase of bars[c]
  int it = blockIdx.x;
  if constexpr (NB == 1) {
    // single buffer: stage the tile, wait, compute, then the next tile
    for (; it < ntiles; it += gridDim.x) {
      stage_begin<T, G, TX, TY>(b, it, pr, stage0, &bars[0], tid, NT);
      const TileRef t = decode_tile<TX, TY>(b, it);
      const InstDev& I = b.inst[t.inst];
      if (I.tma) {
        const unsigned par = phase & 1u;
        const bool ok = mbar_wait(&bars[0], par);
        phase ^= 1u;
        if (__syncthreads_or(!ok)) {
          // the copy did not complete: report, give it one more bounded wait, stop
          if (tid == 0) atomicOr(b.err, 2u);
          mbar_wait(&bars[0], par);
          return;
        }
        if (tile_on_edge<G>(I, t.x0, t.y0)) stage_edges<T, G>(I, pr, stage0, t.x0, t.y0, tid, NT);
      }
      __syncthreads();
      body(I, t, stage0);
      __syncthreads();
    }
    return;
  }
  if (it < ntiles) stage_begin<T, G, TX, TY>(b, it, pr, stage0, &bars[0], tid, NT);
  for (int cur = 0; it < ntiles; it += gridDim.x, cur ^= 1) {
    const int nxt = it + gridDim.x;
    bool next_tma = false;
    if (nxt < ntiles) {
      next_tma = b.inst[find_inst(b.tile_start, b.counts[3], nxt)].tma != 0;
      stage_begin<T, G, TX, TY>(b, nxt, pr, stage0 + (cur ^ 1) * bstride, &bars[cur ^ 1], tid, NT);
    }
    T* sbuf = stage0 + cur * bstride;
    const TileRef t = decode_tile<TX, TY>(b, it);
    const InstDev& I = b.inst[t.inst];
    if (I.tma) {
      const unsigned par = (phase >> cur) & 1u;
      const bool ok = mbar_wait(&bars[cur], par);
      phase ^= 1u << cur;
      if (__syncthreads_or(!ok)) {
        // a copy did not complete: report, give it and the other buffer's copy one more
        // bounded wait each, stop
        if (tid == 0) atomicOr(b.err, 2u);
        mbar_wait(&bars[cur], par);
        if (next_tma) mbar_wait(&bars[cur ^ 1], (phase >> (cur ^ 1)) & 1u);
        return;
      }
      if (tile_on_edge<G>(I, t.x0, t.y0)) stage_edges<T, G>(I, pr, sbuf, t.x0, t.y0, tid, NT);
    }
    __syncthreads();
    body(I, t, sbuf);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// WENO5 reconstruction from precomputed point data.  P points at the centre
// point of the stencil, st is the stride along the line (negative for the
// right-biased reconstruction, which mirrors the left-biased one).  C holds
// (13/3) (f_{m-1} - 2 f_m + f_{m+1})^2 + 4 eps_W per point: the Jiang-Shu
// indicators and eps_W are both scaled by 4, which leaves the normalised
// weights unchanged and makes (eps_W + beta_k) one FMA from C.  FP64 (FP32 WENO5
// runs in registers, w5_rec_f32).  Returns numerator and denominator of
//   sum_k d_k p_k / s_k  /  sum_k d_k / s_k,   s_k = (eps_W + beta_k)^2,
// multiplied through by s_0 s_1 s_2 so that no division is needed here, and
// written about the centred candidate, p_1 + w_0 (p_0 - p_1) + w_2 (p_2 - p_1): the
// differences are third differences of the stencil, (f_{m-2} - 3 f_{m-1} + 3 f_m -
// f_{m+1})/3 = (l_0 + l_1)/3 and (f_{m-1} - 3 f_m + 3 f_{m+1} - f_{m+2})/6 = (l_1 - l_2)/6
// from the indicators' linear terms l_k, so no candidate but p_1 is formed.  With the
// denominator taken 10 times (A + 6 B + 3 C) and the numerator 30 times, their ratio
// is three times the reconstruction; that 3 joins 1/dx in the flux difference
// (flux_scale).  24 FP64 operations against 29 for the three weighted candidates.
template <typename T>
__device__ __forceinline__ void w5_nd(const T* P, const T* C, int st, T& num, T& den) {
  static_assert(std::is_same<T, double>::value, "FP64 reconstruction");
  const T a = P[-2 * st], b = P[-st], c = P[0], d = P[st], e = P[2 * st];
  const T l0 = a - T(4) * b + T(3) * c;
  const T l1 = b - d;
  const T l2 = T(3) * c - T(4) * d + e;
  const T e0 = C[-st] + l0 * l0;
  const T e1 = C[0] + l1 * l1;
  const T e2 = C[st] + l2 * l2;
  const T s0 = e0 * e0, s1 = e1 * e1, s2 = e2 * e2;
  const T A = s1 * s2, B = s0 * s2, Cc = s0 * s1;     // 1 / s_k times s_0 s_1 s_2
  den = fma(T(3), Cc, fma(T(6), B, A));               // 10 (d_0 A + d_1 B + d_2 C)
  const T p1x3 = fma(T(2.5), c, fma(T(-0.5), b, d));  // 3 p_1
  const T ta = l0 + l1, tb = T(1.5) * (l1 - l2);      // 3 (p_0 - p_1), 9 (p_2 - p_1)
  num = fma(p1x3, den, fma(A, ta, Cc * tb));          // 30 (d_0 A p_0 + d_1 B p_1 + d_2 C p_2)
}

// FP32: approximate reciprocal (one MUFU operation, PTX rcp.approx.ftz.f32).
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Interface flux from the left (g+) and right (g-) reconstructions (FP64).
__device__ __forceinline__ double combine(double nl, double dl, double nr, double dr) {
  return (nl * dr + nr * dl) * rcp_newton(dl * dr);
}

// Select a[i] for a small compile-time-sized array without local memory.
template <int N, class P>
__device__ __forceinline__ P pick(const P* a, int i) {
  P r = a[0];
#pragma unroll
  for (int k = 1; k < N; ++k)
    if (i == k) r = a[k];
  return r;
}

// One axis of upwind fluxes for NP flux/partner pairs on the interior lines of
// a staged tile (row stride G::BW).  AX = 0: lines are the TY interior rows,
// points run along x over the W logical columns, TX+1 interfaces per line,
// output [k][row][m].  AX = 1: lines are the TX interior columns, points along
// y over HH rows, TY+1 interfaces per line, output [k][m][col].  The split
// scratch is line-major for AX = 0 and point-major for AX = 1, so that
// neighbouring threads always touch neighbouring words of shared memory.
// g[k], U[k]: staged tiles; NEG bit k negates the flux of pair k.
// split: 4*NP*LS scratch.
template <typename T, int SCHEME, int TX, int TY, int NP, unsigned NEG, int AX>
__device__ __forceinline__ void axis_fluxes(const T* const* g, const T* const* U, T* split, T* out, T ew, int tid) {
  using G = Geo<T, SCHEME, TX, TY>;
  constexpr int H = G::H, W = G::W, HH = G::HH, SW = G::BW, XO = G::XO;
  constexpr int NL = AX == 0 ? TY : TX;           // lines
  constexpr int LL = AX == 0 ? W : HH;            // points per line
  constexpr int NI = AX == 0 ? TX + 1 : TY + 1;   // interfaces per line
  constexpr int LS = NL * LL;
  constexpr int PS = AX == 0 ? 1 : NL;            // split stride between points of a line
  constexpr int NT = TX * TY;
  // index r of the split scratch -> (line, point), and of the interfaces -> (line, m)
  auto pt_line = [&](int r, int& line, int& pt) {
    if (AX == 0) { line = r / LL; pt = r - line * LL; }
    else { pt = r / NL; line = r - pt * NL; }
  };
  auto if_line = [&](int r, int& line, int& m) {
    if (AX == 0) { line = r / NI; m = r - line * NI; }
    else { m = r / NL; line = r - m * NL; }
  };
  auto in_off = [&](int line, int pt) { return AX == 0 ? (H + line) * SW + XO + pt : pt * SW + XO + H + line; };
  auto sp_off = [&](int line, int pt) { return AX == 0 ? line * LL + pt : pt * NL + line; };
  auto out_off = [&](int line, int m) { return AX == 0 ? line * NI + m : m * TX + line; };
  if (SCHEME == LF1_C2) {
    // hat g = (g_m + g_{m+1} - (U_{m+1} - U_m))/2 (Sec. 3.2, alpha = 1)
    for (int k = tid; k < NP * NL * NI; k += NT) {
      const int pr = k / (NL * NI);
      int line, m;
      if_line(k - pr * (NL * NI), line, m);
      const int o0 = in_off(line, H - 1 + m), o1 = in_off(line, H + m);
      const T sg = ((NEG >> pr) & 1u) ? T(-1) : T(1);
      const T* gp = pick<NP>(g, pr);
      const T* up = pick<NP>(U, pr);
      out[pr * NL * NI + out_off(line, m)] = T(0.5) * (sg * gp[o0] + sg * gp[o1] - (up[o1] - up[o0]));
    }
    return;
  }
  // 1. flux splitting g+- = (g +- U)/2 at every point of every line
  for (int k = tid; k < NP * LS; k += NT) {
    const int pr = k / LS, r = k - pr * LS;
    int line, pt;
    pt_line(r, line, pt);
    const int o = in_off(line, pt);
    const T* gp = pick<NP>(g, pr);
    const T gv = ((NEG >> pr) & 1u) ? -gp[o] : gp[o];
    const T uv = pick<NP>(U, pr)[o];
    split[(4 * pr + 0) * LS + r] = gv + uv;   // 2 g+ and 2 g- (the flux comes out doubled)
    split[(4 * pr + 1) * LS + r] = gv - uv;
  }
  __syncthreads();
  if (SCHEME == WENO3_C4) {
    for (int k = tid; k < NP * NL * NI; k += NT) {
      const int pr = k / (NL * NI);
      int line, m;
      if_line(k - pr * (NL * NI), line, m);
      const int c = sp_off(line, H - 1 + m);
      const T* Pp = split + (4 * pr + 0) * LS + c;
      const T* Mm = split + (4 * pr + 1) * LS + c;
      out[pr * NL * NI + out_off(line, m)] =
          weno3<T>(Pp[-PS], Pp[0], Pp[PS], T(4) * ew) + weno3<T>(Mm[2 * PS], Mm[PS], Mm[0], T(4) * ew);
    }
    return;
  }
  if constexpr (SCHEME == WENO5_C4) {
    // 2. curvature part of the smoothness indicators, scaled by 4, plus 4 eps_W (x 4 for the doubled split)
    const T ew4 = T(16) * ew;
    for (int k = tid; k < 2 * NP * LS; k += NT) {
      const int q = k / LS, r = k - q * LS;
      int line, pt;
      pt_line(r, line, pt);
      if (pt == 0 || pt == LL - 1) continue;
      const int pr = q >> 1, pm = q & 1;
      const T* f = split + (4 * pr + pm) * LS + r;
      const T cv = f[-PS] - T(2) * f[0] + f[PS];
      split[(4 * pr + 2 + pm) * LS + r] = T(13.0 / 3.0) * cv * cv + ew4;
    }
    __syncthreads();
    // 3. interface fluxes: left-biased reconstruction of g+ centred at m, right-biased of g- centred at m+1
    for (int k = tid; k < NP * NL * NI; k += NT) {
      const int pr = k / (NL * NI);
      int line, m;
      if_line(k - pr * (NL * NI), line, m);
      const int base = sp_off(line, H - 1 + m);
      T nl, dl, nr, dr;
      w5_nd<T>(split + (4 * pr + 0) * LS + base, split + (4 * pr + 2) * LS + base, PS, nl, dl);
      w5_nd<T>(split + (4 * pr + 1) * LS + base + PS, split + (4 * pr + 3) * LS + base + PS, -PS, nr, dr);
      out[pr * NL * NI + out_off(line, m)] = combine(nl, dl, nr, dr);
    }
  }
}

// FP32 WENO5 fluxes of both axes without shared scratch: a work item is a run
// of KR = 5 consecutive interfaces of one line of one pair (measured faster than
// runs of 3, 4 or 6 on the 16x8 tile: fewer loaded points per interface and
// fewer rounds of items per block).  Its thread loads the KR + 5 points the run
// needs, splits them (g+, g-) and forms their curvature terms in registers,
// then evaluates the interfaces.  Items of the
// x axis come first, then those of the y axis; consecutive threads take
// consecutive lines.  Points past the end of a line are clamped: they only
// feed interfaces of the last run that are not stored.  (Scalar FP32 with
// immediate constants issues fewer instructions here than paired f32x2
// arithmetic, whose operands and constants must first be packed.)

// Scalar FP32 WENO5 reconstruction from register values: the arithmetic of w5_nd
// (about the centred candidate, three times the reconstruction) with reciprocal
// weights r_k = 1 / s_k, as products of the s_k could leave the float range.
__device__ __forceinline__ float w5_rec_f32(float a, float b, float c, float d, float e, float C0, float C1, float C2) {
  const float l0 = fmaf(3.f, c, fmaf(-4.f, b, a));
  const float l1 = b - d;
  const float l2 = fmaf(3.f, c, fmaf(-4.f, d, e));
  const float e0 = fmaf(l0, l0, C0), e1 = fmaf(l1, l1, C1), e2 = fmaf(l2, l2, C2);
  const float r0 = rcp_approx(e0 * e0), r1 = rcp_approx(e1 * e1), r2 = rcp_approx(e2 * e2);
  const float den = fmaf(3.f, r2, fmaf(6.f, r1, r0));          // 10 sum_k d_k r_k
  const float p1x3 = fmaf(2.5f, c, fmaf(-0.5f, b, d));          // 3 p_1
  const float ta = l0 + l1, tb = 1.5f * (l1 - l2);              // 3 (p_0 - p_1), 9 (p_2 - p_1)
  const float num = fmaf(p1x3, den, fmaf(r0, ta, r2 * tb));     // 30 sum_k d_k r_k p_k
  return num * rcp_approx(den);
}

// Values of the LF partner U at a staged point: one plane, or the weighted sum of
// the staged u planes of earlier stages (the explicit-weight dissipation partner),
// summed in stage order.
struct PlaneOne {
  const float* p;
  __device__ __forceinline__ float operator()(int o) const { return p[o]; }
};
struct PlaneSum {
  const float* f[APD_MAXS - 1];
  float w[APD_MAXS - 1];
  int n;
  __device__ __forceinline__ float operator()(int o) const {
    float r = 0.f;
#pragma unroll
    for (int m = 0; m < APD_MAXS - 1; ++m)
      if (m < n) r = r + w[m] * f[m][o];
    return r;
  }
};

#ifndef APD_RUN_LEN
#define APD_RUN_LEN 5   // interfaces per register run
#endif
template <int TX, int TY, int NP, int AX, class UF>
__device__ __forceinline__ void w5_runs_item(const float* g, const UF& U, bool neg, float* out, float ew4, int line,
                                             int run) {
  using G = Geo<float, WENO5_C4, TX, TY>;
  constexpr int H = G::H, SW = G::BW, XO = G::XO, KR = APD_RUN_LEN, NPT = KR + 5;
  constexpr int LL = AX == 0 ? G::W : G::HH;
  constexpr int NI = AX == 0 ? TX + 1 : TY + 1;
  // the last run reads up to point RUNS*KR + 4: inside the staged row for x (BW = TX + 8
  // columns), else clamped to the last row of the line
  constexpr int RUNS = (NI + KR - 1) / KR;
  constexpr bool CLAMP = RUNS * KR + 4 > (AX == 0 ? TX + 6 : LL - 1);
  const int m0 = run * KR;
  float Pp[NPT], Pm[NPT];   // 2 g+ and 2 g- at points m0 .. m0 + KR + 4 of the line (interface m has centre point m + 2)
#pragma unroll
  for (int j = 0; j < NPT; ++j) {
    const int pt = CLAMP ? min(m0 + j, LL - 1) : m0 + j;
    const int o = AX == 0 ? (H + line) * SW + XO + pt : pt * SW + XO + H + line;
    const float gv = neg ? -g[o] : g[o], uv = U(o);
    Pp[j] = gv + uv;
    Pm[j] = gv - uv;
  }
  float Cp[NPT], Cm[NPT];   // (13/3) (f_{j-1} - 2 f_j + f_{j+1})^2 + 16 eps_W (indicators x 4, doubled split)
#pragma unroll
  for (int j = 1; j <= KR + 3; ++j) {
    const float cp = fmaf(-2.f, Pp[j], Pp[j - 1]) + Pp[j + 1];
    const float cm = fmaf(-2.f, Pm[j], Pm[j - 1]) + Pm[j + 1];
    Cp[j] = fmaf(13.f / 3.f * cp, cp, ew4);
    Cm[j] = fmaf(13.f / 3.f * cm, cm, ew4);
  }
#pragma unroll
  for (int i = 0; i < KR; ++i) {
    const int m = m0 + i;
    // left-biased reconstruction of g+ (points m..m+4 of the run), mirrored right-biased of g- (points m+5..m+1)
    const float fl = w5_rec_f32(Pp[i], Pp[i + 1], Pp[i + 2], Pp[i + 3], Pp[i + 4], Cp[i + 1], Cp[i + 2], Cp[i + 3]);
    const float fr = w5_rec_f32(Pm[i + 5], Pm[i + 4], Pm[i + 3], Pm[i + 2], Pm[i + 1], Cm[i + 4], Cm[i + 3], Cm[i + 2]);
    if (NI % KR == 0 || m < NI) out[AX == 0 ? line * NI + m : m * TX + line] = fl + fr;
  }
}

template <int TX, int TY, int NP, unsigned NEGX, unsigned NEGY, class UF>
__device__ __forceinline__ void w5_runs_both_axes(const float* const* gx, const UF* ux, const float* const* gy, const UF* uy,
                                                  float* fx, float* fy, float ew, int tid) {
  constexpr int KR = APD_RUN_LEN, NT = TX * TY;
  constexpr int RX = (TX + 1 + KR - 1) / KR, RY = (TY + 1 + KR - 1) / KR;
  constexpr int IX = NP * TY * RX, IY = NP * TX * RY;
  constexpr int NXI = TY * (TX + 1), NYI = (TY + 1) * TX;
  const float ew4 = 16.f * ew;   // 4 eps_W, x 4 for the doubled split
  for (int k = tid; k < IX + IY; k += NT) {
    if (k < IX) {
      const int pr = k / (TY * RX), r = k - pr * (TY * RX), run = r / TY, line = r - run * TY;
      w5_runs_item<TX, TY, NP, 0>(pick<NP>(gx, pr), pick<NP>(ux, pr), (NEGX >> pr) & 1u, fx + pr * NXI, ew4, line, run);
    } else {
      const int kk = k - IX;
      const int pr = kk / (TX * RY), r = kk - pr * (TX * RY), run = r / TX, line = r - run * TX;
      w5_runs_item<TX, TY, NP, 1>(pick<NP>(gy, pr), pick<NP>(uy, pr), (NEGY >> pr) & 1u, fy + pr * NYI, ew4, line, run);
    }
  }
}

// FP64 WENO5 fluxes of both axes with the passes of the two axes run together:
// the splitting of every point of both axes' lines, then their curvature terms,
// then every interface of both axes, one barrier after each pass.  Merging the
// axes balances the rounds of each pass over the block's threads (the FP64 pipe
// otherwise idles in each pass's last, partly filled round).  The split scratch
// holds both axes: x lines line-major, y lines point-major, as in axis_fluxes.
template <typename T, int TX, int TY, int NP, unsigned NEGX, unsigned NEGY>
__device__ __forceinline__ void w5_fluxes_xy(const T* const* gx, const T* const* ux, const T* const* gy,
                                             const T* const* uy, T* split, T* fx, T* fy, T ew, int tid) {
  using G = Geo<T, WENO5_C4, TX, TY>;
  constexpr int H = G::H, W = G::W, HH = G::HH, SW = G::BW, XO = G::XO, NT = TX * TY;
  constexpr int LSX = G::LSX, LSY = G::LSY, NIX = TX + 1, NIY = TY + 1;
  T* spx = split;                    // [4 NP][LSX]: (row, point)
  T* spy = split + 4 * NP * LSX;     // [4 NP][LSY]: (point, column)
  // 1. flux splitting g+- = (g +- U)/2
  for (int k = tid; k < NP * (LSX + LSY); k += NT) {
    if (k < NP * LSX) {
      const int pr = k / LSX, r = k - pr * LSX, line = r / W, pt = r - line * W;
      const int o = (H + line) * SW + XO + pt;
      const T* gp = pick<NP>(gx, pr);
      const T gv = ((NEGX >> pr) & 1u) ? -gp[o] : gp[o];
      const T uv = pick<NP>(ux, pr)[o];
      spx[(4 * pr + 0) * LSX + r] = gv + uv;   // doubled split, as in axis_fluxes
      spx[(4 * pr + 1) * LSX + r] = gv - uv;
    } else {
      const int kk = k - NP * LSX;
      const int pr = kk / LSY, r = kk - pr * LSY, pt = r / TX, line = r - pt * TX;
      const int o = pt * SW + XO + H + line;
      const T* gp = pick<NP>(gy, pr);
      const T gv = ((NEGY >> pr) & 1u) ? -gp[o] : gp[o];
      const T uv = pick<NP>(uy, pr)[o];
      spy[(4 * pr + 0) * LSY + r] = gv + uv;
      spy[(4 * pr + 1) * LSY + r] = gv - uv;
    }
  }
  __syncthreads();
  // 2. curvature part of the smoothness indicators, scaled by 4, plus 4 eps_W (x 4 for the doubled split)
  const T ew4 = T(16) * ew;
  for (int k = tid; k < 2 * NP * (LSX + LSY); k += NT) {
    if (k < 2 * NP * LSX) {
      const int q = k / LSX, r = k - q * LSX, line = r / W, pt = r - line * W;
      if (pt == 0 || pt == W - 1) continue;
      const int pr = q >> 1, pm = q & 1;
      const T* f = spx + (4 * pr + pm) * LSX + r;
      const T cv = f[-1] - T(2) * f[0] + f[1];
      spx[(4 * pr + 2 + pm) * LSX + r] = T(13.0 / 3.0) * cv * cv + ew4;
    } else {
      const int kk = k - 2 * NP * LSX;
      const int q = kk / LSY, r = kk - q * LSY, pt = r / TX;
      if (pt == 0 || pt == HH - 1) continue;
      const int pr = q >> 1, pm = q & 1;
      const T* f = spy + (4 * pr + pm) * LSY + r;
      const T cv = f[-TX] - T(2) * f[0] + f[TX];
      spy[(4 * pr + 2 + pm) * LSY + r] = T(13.0 / 3.0) * cv * cv + ew4;
    }
  }
  __syncthreads();
  // 3. interface fluxes: left-biased reconstruction of g+ centred at m, right-biased of g- centred at m+1
  for (int k = tid; k < NP * (TY * NIX + TX * NIY); k += NT) {
    T nl, dl, nr, dr;
    if (k < NP * TY * NIX) {
      const int pr = k / (TY * NIX), r = k - pr * (TY * NIX), line = r / NIX, m = r - line * NIX;
      const int base = line * W + (H - 1 + m);
      w5_nd<T>(spx + (4 * pr + 0) * LSX + base, spx + (4 * pr + 2) * LSX + base, 1, nl, dl);
      w5_nd<T>(spx + (4 * pr + 1) * LSX + base + 1, spx + (4 * pr + 3) * LSX + base + 1, -1, nr, dr);
      fx[pr * TY * NIX + line * NIX + m] = combine(nl, dl, nr, dr);
    } else {
      const int kk = k - NP * TY * NIX;
      const int pr = kk / (TX * NIY), r = kk - pr * (TX * NIY), m = r / TX, line = r - m * TX;
      const int base = (H - 1 + m) * TX + line;
      w5_nd<T>(spy + (4 * pr + 0) * LSY + base, spy + (4 * pr + 2) * LSY + base, TX, nl, dl);
      w5_nd<T>(spy + (4 * pr + 1) * LSY + base + TX, spy + (4 * pr + 3) * LSY + base + TX, -TX, nr, dr);
      fy[pr * TX * NIY + m * TX + line] = combine(nl, dl, nr, dr);
    }
  }
}

// Fluxes of both axes for NP pairs: x-axis pairs (gx, ux) into fx [NP][TY][TX+1],
// y-axis pairs (gy, uy) into fy [NP][TY+1][TX].
template <typename T, int SCHEME, int TX, int TY, int NP, unsigned NEGX, unsigned NEGY, bool MERGE = false>
__device__ __forceinline__ void both_axes(const T* const* gx, const T* const* ux, const T* const* gy, const T* const* uy,
                                          T* split, T* fx, T* fy, T ew, int tid) {
  if constexpr (std::is_same<T, float>::value && SCHEME == WENO5_C4) {
    PlaneOne px[NP], py[NP];
#pragma unroll
    for (int k = 0; k < NP; ++k) {
      px[k].p = ux[k];
      py[k].p = uy[k];
    }
    w5_runs_both_axes<TX, TY, NP, NEGX, NEGY>(gx, px, gy, py, fx, fy, ew, tid);
  } else if constexpr (MERGE && SCHEME == WENO5_C4) {
    w5_fluxes_xy<T, TX, TY, NP, NEGX, NEGY>(gx, ux, gy, uy, split, fx, fy, ew, tid);
  } else {
    axis_fluxes<T, SCHEME, TX, TY, NP, NEGX, 0>(gx, ux, split, fx, ew, tid);
    __syncthreads();
    axis_fluxes<T, SCHEME, TX, TY, NP, NEGY, 1>(gy, uy, split, fy, ew, tid);
  }
}

// Planes staged by k_update of stage i: theta, v1, v2 of X^(i), then u1, u2 of
// every earlier stage that enters the dissipation partner.
__device__ __forceinline__ PlaneList update_planes(const BatchDev& b, int i) {
  PlaneList pr;
  pr.add(i, 2);
  pr.add(i, 3);
  pr.add(i, 4);
  for (int jj = 1; jj < i; ++jj)
    if (has(b.m_wp[i], jj)) {
      pr.add(jj, 0);
      pr.add(jj, 1);
    }
  return pr;
}

// Byte sizes of the dynamic shared memory of each kernel (plus 128 for alignment).
template <typename T, int SCHEME, int TX, int TY>
struct StencilSmem {
  using G = Geo<T, SCHEME, TX, TY>;
  static constexpr size_t plane_bytes = sizeof(T) * G::PL;
  static constexpr size_t explicit_bytes = 128 + sizeof(T) * (2 * 6 * G::PL + G::EXPLICIT_EXTRA);
  static constexpr size_t update_fixed_bytes = 128 + sizeof(T) * G::UPDATE_EXTRA;   // + NBUF_U * np * plane_bytes
};

template <typename T>
__device__ __forceinline__ T* aligned_smem(unsigned char* raw) {
  return reinterpret_cast<T*>((reinterpret_cast<uintptr_t>(raw) + 127) & ~uintptr_t(127));
}

// Widening of a transport value to the relaxation's arithmetic type R.  In the FP32
// forms the closed-form relaxations run in FP64 (eps <= 1e-4): their FP32 inputs
// are widened, and their results narrowed, with integer operations (widen_f32,
// narrow_f64_rn: the instructions' results for every class of value) rather than by
// the conversion instructions, which issue on the FP64 pipe, the pipe those kernels'
// FP64 arithmetic already loads (APD_INT_WIDEN = 0 restores the instructions).
#ifndef APD_INT_WIDEN
#define APD_INT_WIDEN 1
#endif
template <typename R, typename T>
__device__ __forceinline__ R widen(T x) {
  if constexpr (APD_INT_WIDEN && std::is_same<R, double>::value && std::is_same<T, float>::value) return widen_f32(x);
  else return R(x);
}
// and the relaxation's result back to the transport type, rounded to nearest
template <typename T, typename R>
__device__ __forceinline__ T narrow(R x) {
  if constexpr (APD_INT_WIDEN && std::is_same<R, double>::value && std::is_same<T, float>::value) return narrow_f64_rn(x);
  else return T(x);
}

// ---------------------------------------------------------------------------
// Closed-form v^(i) at one cell (step 1):
//   v^(i) = (tau eps^2 v^n - dt sum_j atilde_ij E^(j) - dt sum_j a_ij v^(j)) / (tau eps^2 + dt a_ii),
// evaluated in R with the division folded into the coefficients.  E^(jcur)
// and v^(jcur) may be given in registers (the values the kernel has just
// computed or loaded).
template <typename R, typename T>
__device__ __forceinline__ void relax_v_cell(const BatchDev& b, const InstDev& I, int i, size_t o, size_t pl, int jcur,
                                             T ecur1, T ecur2, T vcur1, T vcur2, T& r1, T& r2) {
  const T* Xn = reinterpret_cast<const T*>(I.X);
  const Coef<R>& K = coef<R>(I);
  R a1 = K.r_n[i] * widen<R>(Xn[o + 3 * pl]), a2 = K.r_n[i] * widen<R>(Xn[o + 4 * pl]);
  for (int jj = 1; jj < i; ++jj) {
    if (has(b.m_ex[i], jj)) {
      T e1, e2;
      if (jj == jcur) { e1 = ecur1; e2 = ecur2; }
      else { const T* e = reinterpret_cast<const T*>(I.E[jj]); e1 = e[o]; e2 = e[o + pl]; }
      a1 = a1 + K.rv_e[i][jj] * widen<R>(e1);
      a2 = a2 + K.rv_e[i][jj] * widen<R>(e2);
    }
    if (has(b.m_im[i], jj)) {
      T x1, x2;
      if (jj == jcur) { x1 = vcur1; x2 = vcur2; }
      else { const T* v = reinterpret_cast<const T*>(I.Xs[jj]); x1 = v[o + 3 * pl]; x2 = v[o + 4 * pl]; }
      a1 = a1 + K.rv_v[i][jj] * widen<R>(x1);
      a2 = a2 + K.rv_v[i][jj] * widen<R>(x2);
    }
  }
  r1 = narrow<T>(a1);
  r2 = narrow<T>(a2);
}

// Resident blocks per SM the explicit and update kernels are compiled for: threads worth
// three 256-thread blocks in FP64 (the register budget that removes spills: 128 at 512
// threads), APD_STENCIL_THREADS32 threads in the FP32 forms: 896 (seven 128-thread blocks of
// the 16x8 tile at 72 registers, no spills) measured 8-9 % faster than 768 (six blocks, 80
// registers); 1024 (64 registers) spills.
#ifndef APD_STENCIL_THREADS32
#define APD_STENCIL_THREADS32 896
#endif
#ifndef APD_STENCIL_THREADS64
#define APD_STENCIL_THREADS64 768
#endif
template <typename T>
__host__ __device__ constexpr int stencil_min_blocks(int threads) {
  const int b = (sizeof(T) == 4 ? APD_STENCIL_THREADS32 : APD_STENCIL_THREADS64) / threads;
  return b > 0 ? b : 1;
}

// Factor of 1/h in the difference of interface fluxes: the WENO3 fluxes come out
// doubled (the split without its 1/2), the WENO5 ones six times (the reconstruction
// three times as well); the LF1 flux of Sec. 3.2 comes out as it is.
template <typename T, int SCHEME>
__device__ __forceinline__ T flux_scale(T inv_h) {
  if (SCHEME == LF1_C2) return inv_h;
  if (SCHEME == WENO5_C4) return inv_h * T(1.0 / 6.0);
  return T(0.5) * inv_h;
}

// ---------------------------------------------------------------------------
template <typename T, int SCHEME, int TX, int TY>
__global__ void __launch_bounds__(TX* TY, stencil_min_blocks<T>(TX * TY)) k_explicit(const BatchDev* __restrict__ bp, int j, unsigned need, double weno_eps) {
  using G = Geo<T, SCHEME, TX, TY>;
  constexpr int BW = G::BW, PL = G::PL, NX = G::NX, NY = G::NY;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ uint64_t bars[2];
  T* stage = aligned_smem<T>(smem_raw);   // 2 x 6 planes
  T* split = stage + 2 * 6 * PL;          // 3 pairs
  T* fx = split + 3 * G::SPLIT_PER_PAIR;  // [3][NX]: (q;v1), (-v1;u1), (v2;u2)
  T* fy = fx + 3 * NX;                    // [3][NY]: (q;v2), (v2;u1), (v1;u2)
  const BatchDev& b = *bp;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + ty * TX;
  const T ew = T(weno_eps);
  const bool needB = (need & NEED_DLFB) != 0, needE = (need & NEED_E) != 0;
  PlaneList pr;
  for (int k = 0; k < 6; ++k) pr.add(j, k);
  tile_loop<T, G, TX, TY>(b, pr, stage, bars, tid, [&](const InstDev& I, const TileRef& t, T* s) {
    const T* su1 = s;
    const T* su2 = s + PL;
    const T* sth = s + 2 * PL;
    const T* sv1 = s + 3 * PL;
    const T* sv2 = s + 4 * PL;
    const T* sq = s + 5 * PL;
    const int nx = I.nx;
    const size_t pl = (size_t)nx * I.ny;
    // x-interfaces, then y-interfaces (the split scratch is reused)
    if (needE && needB) {
      const T* gx[3] = {sq, sv1, sv2};
      const T* ux[3] = {sv1, su1, su2};
      const T* gy[3] = {sq, sv2, sv1};
      const T* uy[3] = {sv2, su1, su2};
      both_axes<T, SCHEME, TX, TY, 3, 2u, 0u>(gx, ux, gy, uy, split, fx, fy, ew, tid);
    } else if (needE) {
      const T* gx[1] = {sq};
      const T* ux[1] = {sv1};
      const T* gy[1] = {sq};
      const T* uy[1] = {sv2};
      both_axes<T, SCHEME, TX, TY, 1, 0u, 0u>(gx, ux, gy, uy, split, fx, fy, ew, tid);
    } else if (needB) {
      const T* gx[2] = {sv1, sv2};
      const T* ux[2] = {su1, su2};
      const T* gy[2] = {sv2, sv1};
      const T* uy[2] = {su1, su2};
      both_axes<T, SCHEME, TX, TY, 2, 1u, 0u>(gx, ux, gy, uy, split, fx + NX, fy + NY, ew, tid);
    }
    __syncthreads();
    if (t.x0 + tx >= nx || t.y0 + ty >= I.ny) return;   // beyond the grid (ragged edge tile)
    const Coef<T>& K = coef<T>(I);
    const T idx = K.inv_dx, idy = K.inv_dy;
    const T fidx = flux_scale<T, SCHEME>(idx), fidy = flux_scale<T, SCHEME>(idy);
    const int c = G::C00 + ty * BW + tx;
    const size_t o = (size_t)(t.y0 + ty) * nx + (t.x0 + tx);
    T e1 = T(0), e2 = T(0);
    if (needE) {
      const T b1 = cdiff<T, SCHEME>(su2 + c, BW, idy) - cdiff<T, SCHEME>(su1 + c, 1, idx);
      const T b2 = cdiff<T, SCHEME>(su2 + c, 1, idx) + cdiff<T, SCHEME>(su1 + c, BW, idy);
      const T g1 = (fx[ty * (TX + 1) + tx + 1] - fx[ty * (TX + 1) + tx]) * fidx;
      const T g2 = (fy[(ty + 1) * TX + tx] - fy[ty * TX + tx]) * fidy;
      const T a1 = su1[c], a2 = su2[c];
      const T f1 = T(0.5) * (a2 * a2 - a1 * a1), f2 = a1 * a2;
      const T qt = K.qtau, te2 = K.te2;
      e1 = qt * b1 + te2 * g1 - f1;
      e2 = qt * b2 + te2 * g2 - f2;
      T* e = reinterpret_cast<T*>(I.E[j]);
      e[o] = e1;
      e[o + pl] = e2;
    }
    if (need & NEED_DU) {
      reinterpret_cast<T*>(I.Du[j])[o] = cdiff<T, SCHEME>(su1 + c, 1, idx) + cdiff<T, SCHEME>(su2 + c, BW, idy);
    }
    if (need & NEED_LTH) {
      reinterpret_cast<T*>(I.Lth[j])[o] = cdiff2<T, SCHEME>(sth + c, 1, idx * idx) + cdiff2<T, SCHEME>(sth + c, BW, idy * idy);
    }
    if (needB) {
      // step 3 of every later stage uses D_LF . B(v^(j)) and D_0 theta^(j) only as their
      // sum (times a_ij): one 2-plane field, summed here as it was summed there
      const T* fxb = fx + NX;
      const T* fyb = fy + NY;
      const T d1 = (fxb[ty * (TX + 1) + tx + 1] - fxb[ty * (TX + 1) + tx]) * fidx +
                   (fyb[(ty + 1) * TX + tx] - fyb[ty * TX + tx]) * fidy;
      const T d2 = (fxb[NX + ty * (TX + 1) + tx + 1] - fxb[NX + ty * (TX + 1) + tx]) * fidx +
                   (fyb[NY + (ty + 1) * TX + tx] - fyb[NY + ty * TX + tx]) * fidy;
      T* db = reinterpret_cast<T*>(I.DLFB[j]);
      db[o] = d1 + cdiff<T, SCHEME>(sth + c, 1, idx);
      db[o + pl] = d2 + cdiff<T, SCHEME>(sth + c, BW, idy);
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
  });
}

// ---------------------------------------------------------------------------
// Right-hand side of the Helmholtz equation of stage i (Algorithm 1, step 2; the
// theta-history term with a minus sign, the sign the stage equations of Sec. 3.1 give):
//   R_i = -kappa_i theta^n + sum_{j<i} a_ij/(dt a_ii^2) D_0.u^(j) + 1/(dt a_ii) D_0.u^n
//         - sum_{j<=i} a_ij/a_ii D_0^2:B(v^(j)) - sum_{j<i} a_ij/a_ii D_Delta theta^(j),
// with D_0^2:B(v^(i)) = -D_xx v1 + 2 D_xy v2 + D_yy v1 formed here from v^(i) and stored
// for the later stages.  A work item (rhs_start, rhs_items) is RHS_WARPS consecutive tasks
// of one instance, one per warp: a task is rhs_pairs row pairs times a segment of RHS_SEG
// columns, the warp's lanes holding the columns x0 - 2 .. x0 + RHS_SEG + 1.  A lane loads
// rows y0 - 2 .. y0 + NR + 1 of v1 and v2 at its column once for the task's NR rows, forms
// D_y v2 there, and takes the x-neighbours of v1 and D_y v2 from the neighbouring lanes
// (shuffles): no staging, no barrier but around the per-instance coefficient list and the
// theta sum.  The
// earlier-stage plane terms are summed as (coefficient, plane) pairs from that list in
// one unrolled, predicated loop, all their loads in flight together, before any store.
// The first stage also sums theta^n over the item in a fixed order (th_part).
constexpr int RHS_THREADS = 32 * RHS_WARPS;
// Resident blocks per SM the kernel is compiled for: FP32 7 (72 registers: 0.146 ms per
// step at 2048^2 against 0.151 with 8 blocks at 64; 10 spill; three row pairs per item at
// 6 blocks 0.184), FP64 4 (128 registers: 0.585 ms per step against 0.605 with 5 blocks,
// which spill, and 0.624 with no bound, which takes 136 and runs 3 blocks).
#ifndef APD_RHS_MINB32
#define APD_RHS_MINB32 7
#endif
#ifndef APD_RHS_MINB64
#define APD_RHS_MINB64 4
#endif

template <typename T, int SCHEME>
__global__ void __launch_bounds__(RHS_THREADS, sizeof(T) == 4 ? APD_RHS_MINB32 : APD_RHS_MINB64)
    k_rhs(const BatchDev* __restrict__ bp, int i, double theta_sign, int first_stage) {
  constexpr int MAXT = 1 + 3 * (APD_MAXS - 1);
  constexpr int NR = 2 * rhs_pairs(sizeof(T) == 4);   // rows per item
  constexpr unsigned FULL = 0xffffffffu;
  __shared__ const T* tp[MAXT];
  __shared__ T tc[MAXT];
  __shared__ int s_nt;
  __shared__ double red[RHS_WARPS];
  const BatchDev& b = *bp;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nitems = b.counts[4];
  int cur = -1;   // instance whose coefficient list is in tp, tc
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const int k_inst = find_inst(b.rhs_start, b.counts[3], it);
    const InstDev& I = b.inst[k_inst];
    const Coef<T>& K = coef<T>(I);
    if (k_inst != cur) {
      __syncthreads();   // readers of the previous list are done
      if (tid == 0) {
        const unsigned mim = b.m_im[i];
        int nt = 0;
        auto add = [&](const void* p, T c) {
          tp[nt] = reinterpret_cast<const T*>(p);
          tc[nt++] = c;
        };
        for (int jj = 1; jj < i; ++jj)
          if (has(mim, jj)) add(I.Du[jj], K.c_du[i][jj]);
        add(I.Dun, K.c_dun[i]);
        for (int jj = 1; jj < i; ++jj)
          if (has(mim, jj)) add(I.DB[jj], -K.c_db[i][jj]);
        for (int jj = 1; jj < i; ++jj)
          if (has(mim, jj)) add(I.Lth[jj], theta_sign < 0 ? K.c_lth[i][jj] : -K.c_lth[i][jj]);
        s_nt = nt;
      }
      __syncthreads();
      cur = k_inst;
    }
    const int nt = s_nt;
    const int nx = I.nx, ny = I.ny;
    const size_t pl = (size_t)nx * ny;
    // D_0^2:B(v) = -sx2 S_xx + 2 sx1 S_xy + sy2 S_yy with the unscaled sums S (d1_sum,
    // d2_sum) and D_y v2 = sy1 S_y
    const T sx1 = d1_scale<T, SCHEME>(K.inv_dx), sy1 = d1_scale<T, SCHEME>(K.inv_dy);
    const T msx2 = -d2_scale<T, SCHEME>(K.inv_dx), sy2 = d2_scale<T, SCHEME>(K.inv_dy), sx1x2 = T(2) * sx1;
    const T kap = K.kappa[i];
    const T cdb = has(b.m_im[i], i) ? K.c_db[i][i] : T(0);
    const T* v1 = reinterpret_cast<const T*>(I.Xs[i]) + 3 * pl;
    const T* v2 = v1 + pl;
    const T* th = reinterpret_cast<const T*>(I.X) + 2 * pl;
    T* DBi = reinterpret_cast<T*>(I.DB[i]);
    const bool keep_db = i < b.s;   // D_0^2:B(v^(i)) is read by the later stages only
    T* Rp = reinterpret_cast<T*>(I.R);
    const int local = it - b.rhs_start[k_inst];
    const int nseg = (nx + RHS_SEG - 1) / RHS_SEG;
    const int task = local * RHS_WARPS + warp;          // this warp's (row group, segment)
    const int g = task / nseg, sg = task - g * nseg;
    const int y0 = NR * g, nrows = min(NR, ny - y0);
    const int seg0 = sg * RHS_SEG;                       // first column of this warp's segment
    double tsum = 0.0;
    if (task < rhs_tasks(nx, ny, sizeof(T) == 4)) {   // warp-uniform: past the instance's last task
      const int xs = seg0 + lane - 2;                 // this lane's column, unwrapped
      int x = xs % nx;
      if (x < 0) x += nx;
      const bool outc = lane >= 2 && lane < RHS_SEG + 2 && xs < nx;
      // rows y0 - 2 .. y0 + NR + 1 of v1 and v2 at this lane's column, and the pointwise
      // inputs of the item's rows, all loaded before any store
      T a[NR + 4], c[NR + 4], R[NR], thn[NR];
#pragma unroll
      for (int r = 0; r < NR + 4; ++r) {
        int yy = y0 - 2 + r;
        yy = yy < 0 ? yy + ny : (yy >= ny ? yy - ny : yy);
        const size_t o = (size_t)yy * nx + x;
        a[r] = v1[o];
        c[r] = v2[o];
      }
#pragma unroll
      for (int h = 0; h < NR; ++h) {
        const size_t o = (size_t)(y0 + h) * nx + x;
        const bool on = outc && h < nrows;
        thn[h] = on ? th[o] : T(0);
        T acc = -kap * thn[h];
        if constexpr (sizeof(T) == 8) {
          // FP64: only the terms the stage has (a predicated-off FP64 operation still
          // takes its issue slot on the FP64 pipe)
          if (on)
            for (int t = 0; t < nt; ++t) acc = acc + tc[t] * tp[t][o];
        } else {
#pragma unroll
          for (int t = 0; t < MAXT; ++t)
            if (t < nt && on) acc = acc + tc[t] * tp[t][o];
        }
        R[h] = acc;
      }
#pragma unroll
      for (int h = 0; h < NR; ++h) {
        const T dy = sy1 * d1_sum<T, SCHEME>(c[h], c[h + 1], c[h + 3], c[h + 4]);   // D_y v2 at (x, y0 + h)
        const T v = a[h + 2];
        const T vm1 = __shfl_up_sync(FULL, v, 1), vm2 = __shfl_up_sync(FULL, v, 2);
        const T vp1 = __shfl_down_sync(FULL, v, 1), vp2 = __shfl_down_sync(FULL, v, 2);
        const T dm1 = __shfl_up_sync(FULL, dy, 1), dm2 = __shfl_up_sync(FULL, dy, 2);
        const T dp1 = __shfl_down_sync(FULL, dy, 1), dp2 = __shfl_down_sync(FULL, dy, 2);
        const T sxx = d2_sum<T, SCHEME>(vm2, vm1, v, vp1, vp2);
        const T sxy = d1_sum<T, SCHEME>(dm2, dm1, dp1, dp2);
        const T syy = d2_sum<T, SCHEME>(a[h], a[h + 1], a[h + 2], a[h + 3], a[h + 4]);
        const T Bh = msx2 * sxx + sx1x2 * sxy + sy2 * syy;
        if (outc && h < nrows) {
          const size_t o = (size_t)(y0 + h) * nx + x;
          if (keep_db) DBi[o] = Bh;
          Rp[o] = R[h] - cdb * Bh;
          tsum += double(thn[h]);
        }
      }
    }
    if (first_stage) {
      for (int o = 16; o > 0; o >>= 1) tsum += __shfl_down_sync(FULL, tsum, o);
      if (lane == 0) red[warp] = tsum;
      __syncthreads();
      if (tid == 0) {
        double sum = 0.0;
        for (int w = 0; w < RHS_WARPS; ++w) sum += red[w];
        I.th_part[local] = sum;
      }
      __syncthreads();   // red is rewritten by the next item
    }
  }
}

// ---------------------------------------------------------------------------
template <typename T, int SCHEME, int TX, int TY>
__global__ void __launch_bounds__(TX* TY, stencil_min_blocks<T>(TX * TY)) k_update(const BatchDev* __restrict__ bp, int i, double weno_eps,
                                                                       int close_step, int form) {
  using G = Geo<T, SCHEME, TX, TY>;
  constexpr int BW = G::BW, PL = G::PL, NX = G::NX, NY = G::NY;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ uint64_t bars[2];
  const BatchDev& b = *bp;
  const PlaneList pr = update_planes(b, i);
  const int np = pr.n;
  T* stage = aligned_smem<T>(smem_raw);    // 2 x np planes
  T* sp1 = stage + G::NBUF_U * np * PL;    // dissipation partner (not with register runs)
  T* sp2 = sp1 + PL;
  T* split = G::RUNS ? sp1 : sp2 + PL;     // 2 pairs
  T* fx = split + 2 * G::SPLIT_U_PER_PAIR; // [2][NX]: (-v1;p1), (v2;p2)
  T* fy = fx + 2 * NX;                     // [2][NY]: (v2;p1), (v1;p2)
  const int tx = threadIdx.x, ty = threadIdx.y, tid = tx + ty * TX;
  const T ew = T(weno_eps);
  const unsigned mwp = b.m_wp[i], mim = b.m_im[i];
  tile_loop<T, G, TX, TY, G::NBUF_U>(b, pr, stage, bars, tid, [&](const InstDev& I, const TileRef& t, T* s) {
    const T* sth = s;
    const T* sv1 = s + PL;
    const T* sv2 = s + 2 * PL;
    const int nx = I.nx;
    const size_t pl = (size_t)nx * I.ny;
    // dissipation partner of D_LF . B(v^(i)), the explicit-weight predictor (1/a_ii) sum_{j<i} (atilde_ij - a_ij) u^(j)
    const Coef<T>& K = coef<T>(I);
    if constexpr (G::RUNS) {
      // FP32 WENO5: the register runs form the partner at each point they load
      PlaneSum P1, P2;
      P1.n = P2.n = i - 1;
#pragma unroll
      for (int jj = 1; jj < APD_MAXS; ++jj) {
        const bool on = jj < i && has(mwp, jj);
        const int k = 3 + 2 * __popc(mwp & ((1u << jj) - 2u));      // staged plane of u1^(jj)
        P1.f[jj - 1] = on ? s + k * PL : s;
        P2.f[jj - 1] = on ? s + (k + 1) * PL : s;
        P1.w[jj - 1] = P2.w[jj - 1] = on ? K.wp[i][jj] : 0.f;
      }
      const T* gx[2] = {sv1, sv2};
      const PlaneSum ux[2] = {P1, P2};
      const T* gy[2] = {sv2, sv1};
      const PlaneSum uy[2] = {P1, P2};
      w5_runs_both_axes<TX, TY, 2, 1u, 0u>(gx, ux, gy, uy, fx, fy, ew, tid);
    } else {
      for (int e = tid; e < G::BW * G::BH; e += TX * TY) {
        T p1 = T(0), p2 = T(0);
        int k = 3;
        for (int jj = 1; jj < i; ++jj) {
          if (has(mwp, jj)) {
            p1 = p1 + K.wp[i][jj] * s[k * PL + e];
            p2 = p2 + K.wp[i][jj] * s[(k + 1) * PL + e];
            k += 2;
          }
        }
        sp1[e] = p1;
        sp2[e] = p2;
      }
      __syncthreads();
      const T* gx[2] = {sv1, sv2};
      const T* ux[2] = {sp1, sp2};
      const T* gy[2] = {sv2, sv1};
      const T* uy[2] = {sp1, sp2};
      both_axes<T, SCHEME, TX, TY, 2, 1u, 0u, G::MERGED>(gx, ux, gy, uy, split, fx, fy, ew, tid);
    }
    __syncthreads();
    if (t.x0 + tx >= nx || t.y0 + ty >= I.ny) return;   // beyond the grid (ragged edge tile)
    const T idx = K.inv_dx, idy = K.inv_dy;
    const T fidx = flux_scale<T, SCHEME>(idx), fidy = flux_scale<T, SCHEME>(idy);
    const int c = G::C00 + ty * BW + tx;
    const size_t o = (size_t)(t.y0 + ty) * nx + (t.x0 + tx);
    const T d1 = (fx[ty * (TX + 1) + tx + 1] - fx[ty * (TX + 1) + tx]) * fidx + (fy[(ty + 1) * TX + tx] - fy[ty * TX + tx]) * fidy;
    const T d2 = (fx[NX + ty * (TX + 1) + tx + 1] - fx[NX + ty * (TX + 1) + tx]) * fidx +
                 (fy[NY + (ty + 1) * TX + tx] - fy[NY + ty * TX + tx]) * fidy;
    const T g1 = cdiff<T, SCHEME>(sth + c, 1, idx), g2 = cdiff<T, SCHEME>(sth + c, BW, idy);
    const T dvi = cdiff<T, SCHEME>(sv1 + c, 1, idx) + cdiff<T, SCHEME>(sv2 + c, BW, idy);
    // step 3
    T s1 = T(0), s2 = T(0);
    for (int jj = 1; jj < i; ++jj) {
      if (has(mim, jj)) {
        const T* bg = reinterpret_cast<const T*>(I.DLFB[jj]);   // D_LF . B(v^(jj)) + D_0 theta^(jj)
        s1 = s1 + K.aim[i][jj] * bg[o];
        s2 = s2 + K.aim[i][jj] * bg[o + pl];
      }
    }
    s1 = s1 + K.aim[i][i] * (d1 + g1);
    s2 = s2 + K.aim[i][i] * (d2 + g2);
    const T* Xn = reinterpret_cast<const T*>(I.X);
    T* out = reinterpret_cast<T*>(I.Xs[i]);
    const T dt = K.dt;
    const T u1 = Xn[o] - dt * s1, u2 = Xn[o + pl] - dt * s2;
    if (!close_step) {
      out[o] = u1;
      out[o + pl] = u2;
      reinterpret_cast<T*>(I.Dv[i])[o] = dvi;   // D0 . v^(i) for the q steps of later stages
    }
    // step 4
    T qi;
    if (I.relax64) {
      const Coef<double>& K64 = I.k64;
      double aq = K64.r_n[i] * widen<double>(Xn[o + 5 * pl]);
      for (int jj = 1; jj <= i; ++jj) {
        if (!has(mim, jj)) continue;
        const double dv = widen<double>((jj == i) ? dvi : reinterpret_cast<const T*>(I.Dv[jj])[o]);
        aq = aq + K64.rq_d[i][jj] * dv;
        if (jj < i) aq = aq + K64.rv_v[i][jj] * widen<double>(reinterpret_cast<const T*>(I.Xs[jj])[o + 5 * pl]);
      }
      qi = narrow<T>(aq);
    } else {
      T aq = K.r_n[i] * Xn[o + 5 * pl];
      for (int jj = 1; jj <= i; ++jj) {
        if (!has(mim, jj)) continue;
        const T dv = (jj == i) ? dvi : reinterpret_cast<const T*>(I.Dv[jj])[o];
        aq = aq + K.rq_d[i][jj] * dv;
        if (jj < i) aq = aq + K.rv_v[i][jj] * reinterpret_cast<const T*>(I.Xs[jj])[o + 5 * pl];
      }
      qi = aq;
    }
    if (!close_step) {
      out[o + 5 * pl] = qi;
      return;
    }
    // the close of the step at this cell: X^{n+1} = X^(s) (theta, v of the last stage from the staged tile)
    const T m[6] = {u1, u2, sth[c], sv1[c], sv2[c], qi};
    if (close_step_cell<T>(I, o, pl, m, form, reinterpret_cast<T*>(I.Xnext))) atomicOr(b.err, 1u);
  });
}

}  // namespace apd
