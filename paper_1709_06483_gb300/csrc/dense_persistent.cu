// Dense terms (the long-range spin chain of arXiv:1709.06483, Sec. 4, stored as a dense complex
// matrix): the same persistent Magnus + Leja propagation as leja_persistent.cu (Sec. 2 stepping,
// Sec. 3 Newton recurrence with early termination), with the matvec done for ALL state vectors of
// a row tile at once, so that each Leja iteration reads every dense term exactly once however many
// states share H.  The paper applies dense terms with cuBLAS gemv on one vector (Sec. 3).
//
//  * one vector:  warp per row, lanes stride the columns (coalesced), FP64 FMAs, shuffle reduction;
//  * many vectors: 32-row x 64-vector register tiles over 32-column slices staged in shared memory;
//    every thread owns 2 rows x 4 vectors, each H element read from shared memory serves 4 vectors.
// Both are FP64-pipe bound on GB300 (2 FP64 FMA/clk/SM): a real-valued H x complex state costs 2
// FMAs per element and vector.  A matrix-free sum_i sigma^x_i term may be mixed with dense terms.
//
// Per-vector stop decisions: each block writes its per-vector partial sums; after a barrier every
// block sums each vector's partials over all blocks in the same fixed order, so all blocks hold the
// same totals and take the same decisions.
//
// MAGNUS_TENSOR_SLICED: exact digit products on the tcgen05 tensor cores (dense_tc.cuh), for the
// linear generators and for both product phases of M4 (u_k = H_k w, then the commutators).
#include <math.h>

#include <algorithm>
#include <cuda_bf16.h>

#include "dense_tc.cuh"

#include "magnus_internal.cuh"
#include "persist_common.cuh"

namespace mg {

namespace {

constexpr int kDBlock = 256;
constexpr int kTM = 32;       // rows per tile (tiled path)
constexpr int kTK = 16;       // columns per shared-memory slice
constexpr int kVecMax = 64;   // vectors per tile
constexpr int kPad = 1;

struct DenseSmem {
  double h[kTM][kTK + kPad];            // real parts of coef * H (real-valued terms)
  double hi[kTM][kTK + kPad];           // imaginary parts (complex terms)
  double2 w[kVecMax][kTK + kPad];
};
struct SplitSmem {
  float2 h[kTM][kTK + kPad];            // (hi, lo) of H
  float4 w[kVecMax][kTK + kPad];        // (re_hi, re_lo, im_hi, im_lo) of the vectors
};
union TileSmem {
  DenseSmem d;
  SplitSmem f;
};

// Split-precision multiply-add on the FP32 pipe: sh + sl += (ah + al) (bh + bl).  The leading
// product is exact (TwoProd by FMA), the two cross products are added to its error term, the
// running sum sh is updated by an exact TwoSum, and every rounding error goes to sl.  Explicit
// _rn intrinsics keep the compiler from contracting or reassociating these steps.
__device__ __forceinline__ void df_fma(float ah, float al, float bh, float bl, float &sh, float &sl) {
  const float p = __fmul_rn(ah, bh);
  float e = __fmaf_rn(ah, bh, -p);
  e = __fmaf_rn(ah, bl, e);
  e = __fmaf_rn(al, bh, e);
  const float s = __fadd_rn(sh, p);
  const float z = __fsub_rn(s, sh);
  const float t = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, z)), __fsub_rn(p, z));
  sh = s;
  sl = __fadd_rn(sl, __fadd_rn(t, e));
}

__device__ __forceinline__ float4 split4(double2 v) {
  const float rh = __double2float_rn(v.x), ih = __double2float_rn(v.y);
  return make_float4(rh, __double2float_rn(v.x - (double)rh), ih, __double2float_rn(v.y - (double)ih));
}

// acc[i][q] += coef * sum_j H[r0 + 2 ty + i][j] W[tx + 16 q][j], split precision (see df_fma).
__device__ __forceinline__ void gemm_tile_split(SplitSmem &S, const float2 *H2, double coef, const float4 *W4,
                                                int64_t D, int nv, int64_t r0, int64_t rend, double2 (&acc)[2][4]) {
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  float sh[2][4][2], sl[2][4][2];
#pragma unroll
  for (int i = 0; i < 2; i++)
#pragma unroll
    for (int q = 0; q < 4; q++)
#pragma unroll
      for (int c = 0; c < 2; c++) sh[i][q][c] = sl[i][q][c] = 0.f;
  for (int64_t k0 = 0; k0 < D; k0 += kTK) {
    __syncthreads();
    for (int i = tid; i < kTM * kTK; i += kDBlock) {
      const int rr = i / kTK, kk = i % kTK;
      const int64_t row = r0 + rr, col = k0 + kk;
      S.h[rr][kk] = (row < rend && col < D) ? __ldg(H2 + row * D + col) : make_float2(0.f, 0.f);
    }
    for (int i = tid; i < kVecMax * kTK; i += kDBlock) {
      const int vv = i / kTK, kk = i % kTK;
      const int64_t col = k0 + kk;
      S.w[vv][kk] = (vv < nv && col < D) ? __ldca(W4 + (int64_t)vv * D + col) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();
#pragma unroll 2
    for (int kk = 0; kk < kTK; kk++) {
      const float2 h0 = S.h[2 * ty][kk], h1 = S.h[2 * ty + 1][kk];
#pragma unroll
      for (int q = 0; q < 4; q++) {
        const float4 w = S.w[tx + 16 * q][kk];
        df_fma(h0.x, h0.y, w.x, w.y, sh[0][q][0], sl[0][q][0]);
        df_fma(h0.x, h0.y, w.z, w.w, sh[0][q][1], sl[0][q][1]);
        df_fma(h1.x, h1.y, w.x, w.y, sh[1][q][0], sl[1][q][0]);
        df_fma(h1.x, h1.y, w.z, w.w, sh[1][q][1], sl[1][q][1]);
      }
    }
  }
#pragma unroll
  for (int i = 0; i < 2; i++)
#pragma unroll
    for (int q = 0; q < 4; q++) {
      acc[i][q].x = fma(coef, (double)sh[i][q][0] + (double)sl[i][q][0], acc[i][q].x);
      acc[i][q].y = fma(coef, (double)sh[i][q][1] + (double)sl[i][q][1], acc[i][q].y);
    }
}

// acc[i][q] += sum_j coef * H[r0 + 2 ty + i][j] * W[tx + 16 q][j] over all columns j.
template <bool REAL>
__device__ __forceinline__ void gemm_tile(DenseSmem &S, const Term &T, double coef, const double2 *W, int64_t D,
                                          int nv, int64_t r0, int64_t rend, double2 (&acc)[2][4]) {
  const double2 *H = T.val;
  const double *Hr = T.rv;
  const int64_t rs = T.rs;
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  for (int64_t k0 = 0; k0 < D; k0 += kTK) {
    __syncthreads();
    // stage coef * H[r0 .. r0+31][k0 .. k0+31] (coalesced along the row)
    for (int i = tid; i < kTM * kTK; i += kDBlock) {
      const int rr = i / kTK, kk = i % kTK;
      const int64_t row = r0 + rr, col = k0 + kk;
      if (REAL) {
        S.h[rr][kk] = (row < rend && col < D) ? coef * __ldg(Hr + (row * D + col) * rs) : 0.0;
      } else {
        double2 v = make_double2(0.0, 0.0);
        if (row < rend && col < D) v = __ldg(H + row * D + col);
        S.h[rr][kk] = coef * v.x;
        S.hi[rr][kk] = coef * v.y;
      }
    }
    for (int i = tid; i < kVecMax * kTK; i += kDBlock) {
      const int vv = i / kTK, kk = i % kTK;
      const int64_t col = k0 + kk;
      S.w[vv][kk] = (vv < nv && col < D) ? ldv(W + (int64_t)vv * D + col) : make_double2(0.0, 0.0);
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < kTK; kk++) {
      const double h0 = S.h[2 * ty][kk], h1 = S.h[2 * ty + 1][kk];
      double g0 = 0.0, g1 = 0.0;
      if (!REAL) { g0 = S.hi[2 * ty][kk]; g1 = S.hi[2 * ty + 1][kk]; }
#pragma unroll
      for (int q = 0; q < 4; q++) {
        const double2 wv = S.w[tx + 16 * q][kk];
        acc[0][q] = rfma(h0, wv, acc[0][q]);
        acc[1][q] = rfma(h1, wv, acc[1][q]);
        if (!REAL) {
          acc[0][q].x = fma(-g0, wv.y, acc[0][q].x);
          acc[0][q].y = fma(g0, wv.x, acc[0][q].y);
          acc[1][q].x = fma(-g1, wv.y, acc[1][q].x);
          acc[1][q].y = fma(g1, wv.x, acc[1][q].y);
        }
      }
    }
  }
}

// one row of a dense term times one vector, by a whole warp (lane-strided columns)
template <bool REAL>
__device__ __forceinline__ double2 gemv_row_partial(const Term &T, const double2 *x, int64_t D, int64_t r) {
  const int lane = threadIdx.x & 31;
  double2 acc = make_double2(0.0, 0.0);
  int64_t j = lane;
  if (REAL && T.rs == 1) {  // real storage: 8 B per element
    const double *row = T.rv + r * D;
    for (; j + 96 < D; j += 128) {
      const double a0 = __ldg(row + j), a1 = __ldg(row + j + 32), a2 = __ldg(row + j + 64), a3 = __ldg(row + j + 96);
      const double2 x0 = ldv(x + j), x1 = ldv(x + j + 32), x2 = ldv(x + j + 64), x3 = ldv(x + j + 96);
      acc = rfma(a0, x0, acc); acc = rfma(a1, x1, acc); acc = rfma(a2, x2, acc); acc = rfma(a3, x3, acc);
    }
    for (; j < D; j += 32) acc = rfma(__ldg(row + j), ldv(x + j), acc);
    return acc;
  }
  const double2 *row = T.val + r * D;
  for (; j + 96 < D; j += 128) {
    const double2 a0 = __ldg(row + j), a1 = __ldg(row + j + 32), a2 = __ldg(row + j + 64), a3 = __ldg(row + j + 96);
    const double2 x0 = ldv(x + j), x1 = ldv(x + j + 32), x2 = ldv(x + j + 64), x3 = ldv(x + j + 96);
    if (REAL) {
      acc = rfma(a0.x, x0, acc); acc = rfma(a1.x, x1, acc); acc = rfma(a2.x, x2, acc); acc = rfma(a3.x, x3, acc);
    } else {
      acc = cfma(a0, x0, acc); acc = cfma(a1, x1, acc); acc = cfma(a2, x2, acc); acc = cfma(a3, x3, acc);
    }
  }
  for (; j < D; j += 32) {
    const double2 a0 = __ldg(row + j), x0 = ldv(x + j);
    acc = REAL ? rfma(a0.x, x0, acc) : cfma(a0, x0, acc);
  }
  return acc;  // per-lane partial; caller reduces
}

__device__ __forceinline__ double2 fieldx_at(int n, const double2 *x, int64_t r) {
  double2 acc = make_double2(0.0, 0.0);
  for (int b = 0; b < n; b++) {
    const double2 v = ldv(x + (r ^ ((int64_t)1 << b)));
    acc.x += v.x;
    acc.y += v.y;
  }
  return acc;
}

constexpr int kTcCols = 2 * kVecMax;  // real columns of a vector set: (re, im) of every vector

// exponent e with |x| < 2^e for all |x| <= m (0 for m == 0)
__device__ __forceinline__ int cover_exponent(double m) {
  int e = 0;
  if (m > 0.0) frexp(m, &e);
  return e;
}

// ------------------------------------------------------------------ kernel
// PREC: 0 FP64, 1 FP32 split, 3 digit products on tcgen05 (4 x 8 bits; the product phase of
// dense_tc.cuh, linear generators), 4 the same with M4 (the product phases of u_k = H_k w and of the
// commutators).
constexpr int kEpiTiles = 4;   // 128-row tiles a block's rows can touch (at most 256 rows per block)
constexpr int kEpiOwners = 8;  // CTAs whose partial tiles a tile is summed from

template <bool REAL, bool TILED, int PREC>
__global__ void __launch_bounds__(kDBlock, 1) k_dense_persistent(PersistArgs a) {
  constexpr bool SPLIT = PREC == 1;
  constexpr bool TC = PREC == 3 || PREC == 4;
  constexpr bool TCM4 = PREC == 4;  // tcgen05 with the M4 generator's two product phases
  __shared__ Term sT[kMaxTerms];
  __shared__ ExpRec sR;
  __shared__ double s_vn[kVecMax], s_ep[kVecMax], s_pn[kVecMax];
  __shared__ int s_act[kVecMax], s_m[kVecMax];
  __shared__ double s_part[kDBlock / 32][kVecMax][2];
  __shared__ double s_tot[kVecMax][2];  // per-vector totals of the last reduction
  __shared__ int s_flag;
  __shared__ int s_drift;  // the norm check of the last substep failed
  __shared__ TileSmem TS;
  DenseSmem &S = TS.d;
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ unsigned long long s_cmax[kTcCols];
  __shared__ int s_cexp[kTcCols];
  __shared__ tcg::Bars tc_bars;
  // tcgen05 epilogue: per (dense term, row tile of this block) the offsets of its partial tiles
  __shared__ long long s_own[kMaxTerms][kEpiTiles][kEpiOwners];
  __shared__ int s_nown[kMaxTerms][kEpiTiles];
  __shared__ int s_epi_ok;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ty = tid >> 4, tx = tid & 15;
  const unsigned G = gridDim.x;
  const int b = blockIdx.x;
  const int64_t D = a.dim;
  const int nt = a.nterms, nv = a.nvec;
  // rows of this block: whole tiles (tiled) or any count (one warp per row)
  const int64_t unit = TILED ? kTM : 1;
  const int64_t units = (D + unit - 1) / unit;
  const int64_t per = (units + G - 1) / G;
  const int64_t lo = min(D, (int64_t)b * per * unit), hi = min(D, lo + per * unit);

  for (int i = tid; i < nt * (int)sizeof(Term) / 4; i += blockDim.x)
    reinterpret_cast<int *>(sT)[i] = reinterpret_cast<const int *>(a.terms)[i];
  __syncthreads();
  tcg::Pipe tc_pipe{0u, 0u};
  tcg::Geometry tc_geom{};
  if (TC) {
    tc_geom.ndense = a.tc_ndense;
    tc_geom.T = a.tc_T;
    tc_geom.chunk = tcg::chunk_for(D);
    tc_geom.C = (int)(D / tc_geom.chunk);
    tc_geom.N = a.tc_N;
    tc_geom.slots = a.tc_slots;
    if (tid == 0) {
      for (int i = 0; i < tcg::kNS; i++) {
        tc::mbar_init(&tc_bars.full[i], 1);
        tc::mbar_init(&tc_bars.empty[i], 1);
      }
      tc::mbar_init(&tc_bars.accr, 1);
      tc::mbar_fence_init();
    }
    __syncthreads();
  }

  double *partials = a.partials;                        // [2][G][nv][2]
  unsigned it = 0;
  auto fail = [&](int status) {
    if (tid == 0) atomicCAS(&a.counters->status, 0, status);
  };

  // Reduce per-thread per-vector sums (tiled: vectors tx + 16 q; warp-per-row: the lane's own
  // vector 0) to this block's partials, barrier, every block sums the partials (into s_tot).
  auto reduce_and_share = [&](double (&sw)[4], double (&sp)[4], bool parts_written = false) -> bool {
    double *slot = partials + (size_t)(it & 1u) * G * nv * 2;
    if (parts_written) {  // s_part[warp][v] already holds every warp's share (the tensor-core epilogue)
      __syncthreads();
      for (int v = tid; v < nv; v += blockDim.x) {
        double y0 = 0.0, y1 = 0.0;
        for (int w = 0; w < kDBlock / 32; w++) { y0 += s_part[w][v][0]; y1 += s_part[w][v][1]; }
        slot[((size_t)b * nv + v) * 2] = y0;
        slot[((size_t)b * nv + v) * 2 + 1] = y1;
      }
    } else if (TILED) {
#pragma unroll
      for (int q = 0; q < 4; q++) {
        sw[q] += __shfl_xor_sync(kFull, sw[q], 16);
        sp[q] += __shfl_xor_sync(kFull, sp[q], 16);
      }
      if (lane < 16)
#pragma unroll
        for (int q = 0; q < 4; q++) {
          const int v = tx + 16 * q;
          if (v < nv) { s_part[warp][v][0] = sw[q]; s_part[warp][v][1] = sp[q]; }
        }
      __syncthreads();
      for (int v = tid; v < nv; v += blockDim.x) {
        double y0 = 0.0, y1 = 0.0;
        for (int w = 0; w < kDBlock / 32; w++) { y0 += s_part[w][v][0]; y1 += s_part[w][v][1]; }
        slot[((size_t)b * nv + v) * 2] = y0;
        slot[((size_t)b * nv + v) * 2 + 1] = y1;
      }
    } else {
      if (lane == 0) { s_part[warp][0][0] = sw[0]; s_part[warp][0][1] = sp[0]; }
      __syncthreads();
      if (tid == 0) {
        double y0 = 0.0, y1 = 0.0;
        for (int w = 0; w < kDBlock / 32; w++) { y0 += s_part[w][0][0]; y1 += s_part[w][0][1]; }
        slot[(size_t)b * 2] = y0;
        slot[(size_t)b * 2 + 1] = y1;
      }
    }
    if (!grid_barrier(a.bar, G, a.spin_limit_ns)) return false;
    // every block sums every vector's partials itself, in the same fixed order (warp w takes the
    // vectors w, w + 8, ..., lane l the blocks l, l + 32, ...; the loads of all the warp's vectors go
    // out together): the totals are identical in all blocks and no second barrier is needed
    constexpr int kVpw = kVecMax / (kDBlock / 32);
    double y0[kVpw], y1[kVpw];
#pragma unroll
    for (int i = 0; i < kVpw; i++) y0[i] = y1[i] = 0.0;
    for (int q = lane; q < (int)G; q += 32) {
      double p0[kVpw], p1[kVpw];
#pragma unroll
      for (int i = 0; i < kVpw; i++) {
        const int v = warp + (kDBlock / 32) * i;
        p0[i] = v < nv ? slot[((size_t)q * nv + v) * 2] : 0.0;
        p1[i] = v < nv ? slot[((size_t)q * nv + v) * 2 + 1] : 0.0;
      }
#pragma unroll
      for (int i = 0; i < kVpw; i++) {
        y0[i] += p0[i];
        y1[i] += p1[i];
      }
    }
#pragma unroll
    for (int i = 0; i < kVpw; i++) {
      const int v = warp + (kDBlock / 32) * i;
      const double t0 = warp_sum(y0[i]), t1 = warp_sum(y1[i]);
      if (lane == 0 && v < nv) {
        s_tot[v][0] = t0;
        s_tot[v][1] = t1;
      }
    }
    __syncthreads();
    return true;
  };

  // y[i][q] = sum_k coef_k (H_k src)[row][vec] (+ field), for this thread's outputs
  // tiled: rows r0 + 2 ty + i, vectors tx + 16 q.  warp path: row r, vector 0 (lane 0 holds it).
  // Slicing pass for a vector set X [nv][D] (MAGNUS_TENSOR_SLICED): column maxima of this block's
  // rows -> global atomicMax, barrier, every block derives the same column exponents and writes the
  // digits of its rows, barrier.  Column-maximum slots rotate over three, the one after next is
  // cleared during each pass.
  unsigned slice_ev = 0;
  auto slice_set = [&](const double2 *X, void *digits, int *exps) -> bool {
    unsigned long long *cm = a.colmax + (size_t)(slice_ev % 3u) * kTcCols;
    for (int c = tid; c < kTcCols; c += blockDim.x) s_cmax[c] = 0ull;
    __syncthreads();
    // this block's column maxima: per thread, then per warp (64-bit integer max of the bits of |x|,
    // which orders like |x|), one shared atomic per warp and column
    for (int v = 0; v < nv; v++) {
      unsigned long long m0 = 0ull, m1 = 0ull;
      for (int64_t r = lo + tid; r < hi; r += blockDim.x) {
        const double2 x = X[(int64_t)v * D + r];
        m0 = max(m0, (unsigned long long)__double_as_longlong(fabs(x.x)));
        m1 = max(m1, (unsigned long long)__double_as_longlong(fabs(x.y)));
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        m0 = max(m0, __shfl_xor_sync(kFull, m0, o));
        m1 = max(m1, __shfl_xor_sync(kFull, m1, o));
      }
      if (lane == 0 && (m0 | m1)) {
        atomicMax(&s_cmax[2 * v], m0);
        atomicMax(&s_cmax[2 * v + 1], m1);
      }
    }
    __syncthreads();
    for (int c = tid; c < 2 * nv; c += blockDim.x)
      if (s_cmax[c]) atomicMax(&cm[c], s_cmax[c]);
    if (!grid_barrier(a.bar, G, a.spin_limit_ns)) return false;
    for (int c = tid; c < 2 * nv; c += blockDim.x) {
      s_cexp[c] = cover_exponent(__longlong_as_double((long long)cm[c]));
      if (b == 0) exps[c] = s_cexp[c];
    }
    if (b == 0)
      for (int c = tid; c < kTcCols; c += blockDim.x) a.colmax[(size_t)((slice_ev + 2) % 3u) * kTcCols + c] = 0ull;
    __syncthreads();
    __nv_bfloat16 *dg = (__nv_bfloat16 *)digits;
    // one work item = one column and 8 consecutive rows (this block's rows come in whole 32-row
    // tiles): the digits of the 8 values go out as four 16-byte stores
    const int ncol = 2 * nv;
    const int64_t ngroups = (hi - lo) / 8;
    for (int64_t w = tid; w < ngroups * ncol; w += blockDim.x) {
      const int c = (int)(w % ncol), v = c >> 1;
      const int64_t r0 = lo + 8 * (w / ncol);
      double xv[8];
#pragma unroll
      for (int i = 0; i < 8; i++) {
        const double2 x = X[(int64_t)v * D + r0 + i];
        xv[i] = (c & 1) ? x.y : x.x;
      }
      tcg::slice8_tiled(xv, s_cexp[c], dg, D, c, r0);
    }
    // the digits are read next by TMA (async proxy) in other CTAs
    asm volatile("fence.proxy.async.global;" ::: "memory");
    slice_ev++;
    return grid_barrier(a.bar, G, a.spin_limit_ns);
  };

  // tcgen05 path: vector set s of the digit buffer and its column exponents
  auto tc_set_digits = [&](int set) { return (void *)((__nv_bfloat16 *)a.tc_wd + (size_t)set * tcg::kSl * tcg::kN * D); };
  auto tc_set_exps = [&](int set) { return a.tc_ex + set * kTcCols; };
  // y += coef (H_k W)[rows of this 32-row tile] from the partial tiles of the last product phase
  auto tc_term = [&](int k, double coef, int64_t r0, double2 (&y)[2][4]) {
#pragma unroll
    for (int i = 0; i < 2; i++) {
      const int64_t r = r0 + 2 * ty + i;
      if (r >= hi) continue;
      const long long tile = (long long)a.tc_dslot[k] * tc_geom.T + r / tcg::kM;
      const int rr = (int)(r % tcg::kM);
      int bf, bl;
      tcg::tile_owners(tile, tc_geom, (int)G, &bf, &bl);
      double sx[4] = {0.0, 0.0, 0.0, 0.0}, sy[4] = {0.0, 0.0, 0.0, 0.0};
      for (int bb = bf; bb <= bl; bb++) {  // the CTAs holding chunks of this tile, in order
        const long long b_lo = tcg::range_lo(bb, (int)G, tc_geom.N);
        if (b_lo == tcg::range_lo(bb + 1, (int)G, tc_geom.N)) continue;
        const double *Pt = a.tc_P + ((size_t)bb * tc_geom.slots + (size_t)(tile - b_lo / tc_geom.C)) *
                                        (size_t)(tcg::kN * tcg::kM) + rr;
#pragma unroll
        for (int q = 0; q < 4; q++) {
          const int v = tx + 16 * q;
          if (v < nv) {
            sx[q] += Pt[(size_t)(2 * v) * tcg::kM];
            sy[q] += Pt[(size_t)(2 * v + 1) * tcg::kM];
          }
        }
      }
#pragma unroll
      for (int q = 0; q < 4; q++) {
        y[i][q].x = fma(coef, sx[q], y[i][q].x);
        y[i][q].y = fma(coef, sy[q], y[i][q].y);
      }
    }
  };

  // the sets of one product phase: every dense term multiplies set `set`
  auto tc_all = [&](int set) {
    tcg::Sets W;
    for (int q = 0; q < tcg::kMaxSets; q++) {
      W.wd[q] = (const __nv_bfloat16 *)tc_set_digits(set);
      W.ec[q] = tc_set_exps(set);
    }
    return W;
  };
  // one product phase on the tensor cores (this CTA's items), then a barrier
  auto tc_products = [&](const tcg::Sets &W) -> bool {
    if (!tcg::gemm_phase((const __nv_bfloat16 *)a.tc_hd, W, tc_geom, a.tc_eh, a.tc_P, dsm, tc_bars, tc_pipe,
                         a.tc_spins))
      return false;
    return grid_barrier(a.bar, G, a.spin_limit_ns);
  };

  auto apply_terms = [&](const double *coef, const double2 *const *srcs, const float4 *const *shs, int64_t r0,
                         double2 (&y)[2][4]) {
    if (TILED) {
#pragma unroll
      for (int i = 0; i < 2; i++)
#pragma unroll
        for (int q = 0; q < 4; q++) y[i][q] = make_double2(0.0, 0.0);
      for (int k = 0; k < nt; k++) {
        if (coef[k] == 0.0) continue;
        if (sT[k].kind == MAGNUS_TERM_DENSE) {
          if (TC)
            tc_term(k, coef[k], r0, y);
          else if (SPLIT)
            gemm_tile_split(TS.f, a.hsplit[k], coef[k], shs[k], D, nv, r0, hi, y);
          else
            gemm_tile<REAL>(S, sT[k], coef[k], srcs[k], D, nv, r0, hi, y);
        } else if (sT[k].kind == MAGNUS_TERM_FIELD_X) {
#pragma unroll
          for (int i = 0; i < 2; i++) {
            const int64_t r = r0 + 2 * ty + i;
            if (r >= hi) continue;
#pragma unroll
            for (int q = 0; q < 4; q++) {
              const int v = tx + 16 * q;
              if (v < nv) y[i][q] = rfma(coef[k], fieldx_at(sT[k].nspins, srcs[k] + (int64_t)v * D, r), y[i][q]);
            }
          }
        }
      }
    } else {
      double2 acc = make_double2(0.0, 0.0);
      for (int k = 0; k < nt; k++) {
        if (coef[k] == 0.0) continue;
        if (sT[k].kind == MAGNUS_TERM_DENSE) {
          const double2 part = gemv_row_partial<REAL>(sT[k], srcs[k], D, r0);
          acc = rfma(coef[k], part, acc);
        } else if (sT[k].kind == MAGNUS_TERM_FIELD_X && lane == 0) {
          acc = rfma(coef[k], fieldx_at(sT[k].nspins, srcs[k], r0), acc);
        }
      }
      acc.x = warp_sum(acc.x);
      acc.y = warp_sum(acc.y);
      y[0][0] = acc;
    }
  };

  // ||psi|| of every vector
  {
    double sw[4] = {0, 0, 0, 0}, sp[4] = {0, 0, 0, 0};
    if (TILED) {
      for (int64_t r0 = lo; r0 < hi; r0 += kTM)
        for (int i = 0; i < 2; i++) {
          const int64_t r = r0 + 2 * ty + i;
          if (r >= hi) continue;
          for (int q = 0; q < 4; q++) {
            const int v = tx + 16 * q;
            if (v < nv) sw[q] += cabs2(a.psi[(int64_t)v * D + r]);
          }
        }
    } else {
      for (int64_t r = lo + tid; r < hi; r += blockDim.x) sw[0] += cabs2(a.psi[r]);
      sw[0] = warp_sum(sw[0]);
    }
    if (!reduce_and_share(sw, sp)) { fail(MAGNUS_ETIMEOUT); return; }
    if (tid < nv) s_vn[tid] = sqrt(s_tot[tid][0]);
    __syncthreads();
    it++;
  }

  double2 *cur = a.psi, *nxt = a.alt;
  long long sub_counter = 0;
  for (int64_t e = 0; e < a.nexp; e++) {
    __syncthreads();
    if (tid == 0) sR = a.recs[e];
    __syncthreads();
    const ExpRec &R = sR;
    const double2 *d = a.dd + e * (int64_t)(a.m_max + 1);
    if (!(R.gamma > 0.0)) {
      const double2 ph = d[0];
      for (int v = 0; v < nv; v++)
        for (int64_t r = lo + tid; r < hi; r += blockDim.x) nxt[(int64_t)v * D + r] = cmul(ph, cur[(int64_t)v * D + r]);
      if (!grid_barrier(a.bar, G, a.spin_limit_ns)) { fail(MAGNUS_ETIMEOUT); return; }
      double2 *tmp = cur; cur = nxt; nxt = tmp;
      if (b == 0 && tid == 0) a.counters->n_exp++;
      continue;
    }
    const double2 d0 = d[0];
    for (int sub = 0; sub < R.s; sub++) {
      if (tid < nv) {
        s_act[tid] = 1;
        s_ep[tid] = sqrt(cabs2(d0)) * s_vn[tid];
        s_m[tid] = 0;
      }
      if (SPLIT) {  // split copy of the substep's input vector, read by every block
        for (int v = 0; v < nv; v++)
          for (int64_t r = lo + tid; r < hi; r += blockDim.x)
            a.sh_cur[(int64_t)v * D + r] = split4(cur[(int64_t)v * D + r]);
        if (!grid_barrier(a.bar, G, a.spin_limit_ns)) { fail(MAGNUS_ETIMEOUT); return; }
      }
      if (TC) {
        if (!slice_set(cur, tc_set_digits(0), tc_set_exps(0))) { fail(MAGNUS_ETIMEOUT); return; }
      }
      __syncthreads();
      bool done = false;
      for (int j = 1; j <= a.m_max; j++) {
        const double2 *src = (j == 1) ? cur : (((j - 2) & 1) ? a.w1 : a.w0);
        double2 *dst = ((j - 1) & 1) ? a.w1 : a.w0;
        const float4 *src_sh = (j == 1) ? a.sh_cur : (((j - 2) & 1) ? a.sh_w1 : a.sh_w0);
        float4 *dst_sh = ((j - 1) & 1) ? a.sh_w1 : a.sh_w0;
        const double shift = R.cg + a.xi[j - 1];
        const double2 dj = d[j];
        const double2 *srcs[kMaxTerms] = {src, src, src, src};
        const float4 *shs[kMaxTerms] = {src_sh, src_sh, src_sh, src_sh};
        if (TC) {  // all dense products of this iteration on the tensor cores, then a barrier
          if (!TCM4 && R.mode != MODE_LINEAR) { fail(MAGNUS_EINVAL); return; }
          const int set = (j == 1) ? 0 : (((j - 2) & 1) ? 2 : 1);
          if (!tc_products(tc_all(set))) { fail(MAGNUS_ETIMEOUT); return; }
        }
        if ((!TC || TCM4) && R.mode == MODE_M4) {
          // phase 1: u_k = H_k src for every vector, this block's rows
          double one[kMaxTerms];
          for (int k = 0; k < nt; k++) {
            for (int q = 0; q < kMaxTerms; q++) one[q] = (q == k) ? 1.0 : 0.0;
            double2 *uk = a.u + (size_t)k * nv * D;
            if (TILED) {
              for (int64_t r0 = lo; r0 < hi; r0 += kTM) {
                double2 y[2][4];
                apply_terms(one, srcs, shs, r0, y);
                for (int i = 0; i < 2; i++) {
                  const int64_t r = r0 + 2 * ty + i;
                  if (r >= hi) continue;
                  for (int q = 0; q < 4; q++) {
                    const int v = tx + 16 * q;
                    if (v < nv) {
                      uk[(int64_t)v * D + r] = y[i][q];
                      if (SPLIT) a.sh_u[(size_t)k * nv * D + (int64_t)v * D + r] = split4(y[i][q]);
                    }
                  }
                }
              }
            } else {
              for (int64_t r = lo + warp; r < hi; r += kDBlock / 32) {
                double2 y[2][4];
                apply_terms(one, srcs, shs, r, y);
                if (lane == 0) uk[r] = y[0][0];
              }
            }
          }
          if (!grid_barrier(a.bar, G, a.spin_limit_ns)) { fail(MAGNUS_ETIMEOUT); return; }
          if (TCM4)  // digits of every u_k: set 3 + k
            for (int k = 0; k < nt; k++)
              if (!slice_set(a.u + (size_t)k * nv * D, tc_set_digits(3 + k), tc_set_exps(3 + k))) {
                fail(MAGNUS_ETIMEOUT);
                return;
              }
        }
        double sw[4] = {0, 0, 0, 0}, sp[4] = {0, 0, 0, 0};
        // epilogue for one output (row r, vector v) with y = the combined matvec
        // tcgen05 path: column maxima of the new w_j, gathered here for the next slicing pass
        unsigned long long cmx[4] = {0ull, 0ull, 0ull, 0ull}, cmy[4] = {0ull, 0ull, 0ull, 0ull};
        auto finish = [&](int64_t r, int v, double2 y, int q) {
          const int64_t idx = (int64_t)v * D + r;
          const double2 wr = ldv(src + idx);
          y = rfma(-shift, wr, y);
          dst[idx] = y;
          if (TC) {
            cmx[q] = max(cmx[q], (unsigned long long)__double_as_longlong(fabs(y.x)));
            cmy[q] = max(cmy[q], (unsigned long long)__double_as_longlong(fabs(y.y)));
          }
          if (SPLIT) dst_sh[idx] = split4(y);
          double2 pr = (j == 1) ? cmul(d0, wr) : nxt[idx];
          pr = cfma(dj, y, pr);
          nxt[idx] = pr;
          sw[q] += cabs2(y);
          sp[q] += cabs2(pr);
        };
        // y += -i kg (H_k u_l - H_l u_k) for one pair k < l, this thread's outputs of the tile at r0
        auto comm_pair = [&](int k, int l, double kg, int64_t r0, double2 (&y)[2][4]) {
          double ck[kMaxTerms] = {0, 0, 0, 0}, cl[kMaxTerms] = {0, 0, 0, 0};
          ck[k] = kg;
          cl[l] = -kg;
          const double2 *sk[kMaxTerms], *sl[kMaxTerms];
          const float4 *hk[kMaxTerms], *hl[kMaxTerms];
          for (int q = 0; q < kMaxTerms; q++) {
            sk[q] = a.u + (size_t)l * nv * D;  // H_k applied to u_l
            sl[q] = a.u + (size_t)k * nv * D;  // H_l applied to u_k
            hk[q] = a.sh_u + (size_t)l * nv * D;
            hl[q] = a.sh_u + (size_t)k * nv * D;
          }
          double2 z1[2][4], z2[2][4];
          apply_terms(ck, sk, hk, r0, z1);
          apply_terms(cl, sl, hl, r0, z2);
          for (int i = 0; i < 2; i++)
            for (int q = 0; q < 4; q++) {
              const double zx = z1[i][q].x + z2[i][q].x, zy = z1[i][q].y + z2[i][q].y;
              y[i][q].x += zy;  // -i z
              y[i][q].y -= zx;
            }
        };
        auto commutator = [&](int64_t r0, double2 (&y)[2][4]) {
          // y += -i sum_{k<l} kg_kl (H_k u_l - H_l u_k)
          int pi = 0;
          for (int k = 0; k < nt; k++)
            for (int l = k + 1; l < nt; l++, pi++)
              if (R.kg[pi] != 0.0) comm_pair(k, l, R.kg[pi], r0, y);
        };
        if (TCM4 && R.mode == MODE_M4) {
          // the commutators on the tensor cores: per pair k < l one product phase in which dense term
          // k multiplies the digits of u_l and dense term l those of u_k; -i kg (H_k u_l - H_l u_k) of
          // the pairs, in pair order, summed into tc_cacc for this block's rows (the order of the
          // commutator above, so the same sums)
          int pi = 0;
          bool first = true;
          for (int k = 0; k < nt; k++)
            for (int l = k + 1; l < nt; l++, pi++) {
              if (R.kg[pi] == 0.0) continue;
              const bool dk = sT[k].kind == MAGNUS_TERM_DENSE, dl = sT[l].kind == MAGNUS_TERM_DENSE;
              if (dk || dl) {
                // every block has summed the previous phase's partial tiles before they are rewritten
                if (!first && !grid_barrier(a.bar, G, a.spin_limit_ns)) { fail(MAGNUS_ETIMEOUT); return; }
                tcg::Sets W = tc_all(3 + l);
                if (dl) {
                  W.wd[a.tc_dslot[l]] = (const __nv_bfloat16 *)tc_set_digits(3 + k);
                  W.ec[a.tc_dslot[l]] = tc_set_exps(3 + k);
                }
                if (!tc_products(W)) { fail(MAGNUS_ETIMEOUT); return; }
              }
              for (int64_t r0 = lo; r0 < hi; r0 += kTM) {
                double2 z[2][4];
                for (int i = 0; i < 2; i++)
                  for (int q = 0; q < 4; q++) {
                    const int64_t r = r0 + 2 * ty + i;
                    const int v = tx + 16 * q;
                    z[i][q] = (first || r >= hi || v >= nv) ? make_double2(0.0, 0.0) : a.tc_cacc[(int64_t)v * D + r];
                  }
                comm_pair(k, l, R.kg[pi], r0, z);
                for (int i = 0; i < 2; i++)
                  for (int q = 0; q < 4; q++) {
                    const int64_t r = r0 + 2 * ty + i;
                    const int v = tx + 16 * q;
                    if (r < hi && v < nv) a.tc_cacc[(int64_t)v * D + r] = z[i][q];
                  }
              }
              first = false;
            }
          if (first)  // no commutator
            for (int v = 0; v < nv; v++)
              for (int64_t r = lo + tid; r < hi; r += blockDim.x) a.tc_cacc[(int64_t)v * D + r] = make_double2(0.0, 0.0);
          __syncthreads();
        }
        bool tc_epi = false;
        const int64_t t_first = lo / tcg::kM;  // first 128-row tile of this block's rows
        if (TC && R.mode == MODE_LINEAR) {
          // epilogue of the tensor-core products: warp w takes the vectors w, w + 8, ..., its lanes
          // the block's rows, so that the partial tiles (row-contiguous per column) and the vectors
          // are read and written in consecutive runs.  y sums the terms in term order and each
          // tile's owners in CTA order, as tc_term does.
          // the CTAs holding each (dense term, 128-row tile) of this block's rows and the offsets of
          // their partial tiles, in CTA order: a small table made once per iteration (the general
          // path below serves blocks whose rows or tiles do not fit it)
          if (tid == 0) s_epi_ok = (hi <= lo) || ((hi - 1) / tcg::kM - t_first < kEpiTiles);
          __syncthreads();
          if (tid < kMaxTerms * kEpiTiles && s_epi_ok) {
            const int k = tid / kEpiTiles, ti = tid % kEpiTiles;
            int n_own = 0;
            const int64_t rt = t_first + ti;
            if (k < nt && sT[k].kind == MAGNUS_TERM_DENSE && lo < hi && rt * tcg::kM < hi) {
              const long long tile = (long long)a.tc_dslot[k] * tc_geom.T + rt;
              int bf, bl;
              tcg::tile_owners(tile, tc_geom, (int)G, &bf, &bl);
              for (int bb = bf; bb <= bl; bb++) {
                const long long b_lo = tcg::range_lo(bb, (int)G, tc_geom.N);
                if (b_lo == tcg::range_lo(bb + 1, (int)G, tc_geom.N)) continue;
                if (n_own == kEpiOwners) {
                  s_epi_ok = 0;  // more owners than the table holds (benign race: every writer stores 0)
                  break;
                }
                s_own[k][ti][n_own++] = ((long long)bb * tc_geom.slots + (tile - b_lo / tc_geom.C)) *
                                        (long long)(tcg::kN * tcg::kM);
              }
            }
            s_nown[k][ti] = n_own;
          }
          for (int v = lane; v < kVecMax; v += 32) {
            s_part[warp][v][0] = 0.0;
            s_part[warp][v][1] = 0.0;
          }
          __syncthreads();
          tc_epi = s_epi_ok != 0;
        }
        if (tc_epi) {
          // y[r][v] = sum_k coef_k (H_k W)[r][v] (+ field terms), terms in order, owners in CTA order
          auto epi_y = [&](int64_t r, int v) {
            double2 y = make_double2(0.0, 0.0);
            const int ti = (int)(r / tcg::kM - t_first), rr = (int)(r % tcg::kM);
            for (int k = 0; k < nt; k++) {
              const double coef = R.bg[k];
              if (coef == 0.0) continue;
              if (sT[k].kind == MAGNUS_TERM_DENSE) {
                double sx = 0.0, sy = 0.0;
                const int no = s_nown[k][ti];
                for (int o = 0; o < no; o++) {
                  const double *Pt = a.tc_P + s_own[k][ti][o] + rr;
                  sx += Pt[(size_t)(2 * v) * tcg::kM];
                  sy += Pt[(size_t)(2 * v + 1) * tcg::kM];
                }
                y.x = fma(coef, sx, y.x);
                y.y = fma(coef, sy, y.y);
              } else if (sT[k].kind == MAGNUS_TERM_FIELD_X) {
                y = rfma(coef, fieldx_at(sT[k].nspins, src + (int64_t)v * D, r), y);
              }
            }
            return y;
          };
          for (int v = warp; v < nv; v += kDBlock / 32) {
            double pw = 0.0, pp = 0.0;
            unsigned long long mx = 0ull, my = 0ull;
            if (s_act[v])
              for (int64_t r0 = lo; r0 < hi; r0 += 64) {  // two rows per lane, their loads together
                const int64_t ra = r0 + lane, rb = r0 + 32 + lane;
                const bool ia = ra < hi, ib = rb < hi;
                double2 ya = make_double2(0.0, 0.0), yb = ya, wa = ya, wb = ya, pa = ya, pb = ya;
                const int64_t xa = (int64_t)v * D + ra, xb = (int64_t)v * D + rb;
                if (ia) { ya = epi_y(ra, v); wa = ldv(src + xa); if (j > 1) pa = nxt[xa]; }
                if (ib) { yb = epi_y(rb, v); wb = ldv(src + xb); if (j > 1) pb = nxt[xb]; }
                if (ia) {
                  ya = rfma(-shift, wa, ya);
                  dst[xa] = ya;
                  mx = max(mx, (unsigned long long)__double_as_longlong(fabs(ya.x)));
                  my = max(my, (unsigned long long)__double_as_longlong(fabs(ya.y)));
                  pa = cfma(dj, ya, (j == 1) ? cmul(d0, wa) : pa);
                  nxt[xa] = pa;
                  pw += cabs2(ya);
                  pp += cabs2(pa);
                }
                if (ib) {
                  yb = rfma(-shift, wb, yb);
                  dst[xb] = yb;
                  mx = max(mx, (unsigned long long)__double_as_longlong(fabs(yb.x)));
                  my = max(my, (unsigned long long)__double_as_longlong(fabs(yb.y)));
                  pb = cfma(dj, yb, (j == 1) ? cmul(d0, wb) : pb);
                  nxt[xb] = pb;
                  pw += cabs2(yb);
                  pp += cabs2(pb);
                }
              }
            pw = warp_sum(pw);
            pp = warp_sum(pp);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
              mx = max(mx, __shfl_xor_sync(kFull, mx, o));
              my = max(my, __shfl_xor_sync(kFull, my, o));
            }
            if (lane == 0) {
              s_part[warp][v][0] = pw;
              s_part[warp][v][1] = pp;
              s_cmax[2 * v] = mx;
              s_cmax[2 * v + 1] = my;
            }
          }
        } else if (TILED) {
          for (int64_t r0 = lo; r0 < hi; r0 += kTM) {
            double2 y[2][4];
            if (R.mode == MODE_M4) {
              for (int i = 0; i < 2; i++)
                for (int q = 0; q < 4; q++) {
                  const int64_t r = r0 + 2 * ty + i;
                  const int v = tx + 16 * q;
                  y[i][q] = (TCM4 && r < hi && v < nv) ? a.tc_cacc[(int64_t)v * D + r] : make_double2(0.0, 0.0);
                }
              if (!TC) commutator(r0, y);
              for (int i = 0; i < 2; i++) {
                const int64_t r = r0 + 2 * ty + i;
                if (r >= hi) continue;
                for (int q = 0; q < 4; q++) {
                  const int v = tx + 16 * q;
                  if (v >= nv) continue;
                  for (int k = 0; k < nt; k++) y[i][q] = rfma(R.bg[k], a.u[(size_t)k * nv * D + (int64_t)v * D + r], y[i][q]);
                }
              }
            } else {
              apply_terms(R.bg, srcs, shs, r0, y);
            }
            for (int i = 0; i < 2; i++) {
              const int64_t r = r0 + 2 * ty + i;
              if (r >= hi) continue;
              for (int q = 0; q < 4; q++) {
                const int v = tx + 16 * q;
                if (v < nv && s_act[v]) finish(r, v, y[i][q], q);
              }
            }
          }
        } else {
          for (int64_t r = lo + warp; r < hi; r += kDBlock / 32) {
            double2 y[2][4];
            if (R.mode == MODE_M4) {
              y[0][0] = make_double2(0.0, 0.0);
              commutator(r, y);
              for (int k = 0; k < nt; k++) y[0][0] = rfma(R.bg[k], a.u[(size_t)k * D + r], y[0][0]);
            } else {
              apply_terms(R.bg, srcs, shs, r, y);
            }
            if (lane == 0 && s_act[0]) finish(r, 0, y[0][0], 0);
          }
        }
        if (!TILED) sw[0] = warp_sum(sw[0]), sp[0] = warp_sum(sp[0]);
        if (tc_epi && j < a.m_max) {  // this block's column maxima (written above) -> the epilogue slot
          __syncthreads();
          for (int c = tid; c < 2 * nv; c += blockDim.x)
            if (s_cmax[c]) atomicMax(&a.colmax[3 * kTcCols + c], s_cmax[c]);
        } else if (TC && j < a.m_max) {  // this block's column maxima -> the epilogue slot (published by the next barrier)
          for (int c = tid; c < kTcCols; c += blockDim.x) s_cmax[c] = 0ull;
          __syncthreads();
#pragma unroll
          for (int q = 0; q < 4; q++) {
            cmx[q] = max(cmx[q], __shfl_xor_sync(kFull, cmx[q], 16));
            cmy[q] = max(cmy[q], __shfl_xor_sync(kFull, cmy[q], 16));
          }
          if (lane < 16)
#pragma unroll
            for (int q = 0; q < 4; q++) {
              const int v = tx + 16 * q;
              if (v < nv) {
                if (cmx[q]) atomicMax(&s_cmax[2 * v], cmx[q]);
                if (cmy[q]) atomicMax(&s_cmax[2 * v + 1], cmy[q]);
              }
            }
          __syncthreads();
          for (int c = tid; c < 2 * nv; c += blockDim.x)
            if (s_cmax[c]) atomicMax(&a.colmax[3 * kTcCols + c], s_cmax[c]);
        }
        if (!reduce_and_share(sw, sp, tc_epi)) { fail(MAGNUS_ETIMEOUT); return; }
        if (warp == 0) {  // every vector's stop test, one lane per vector (they are independent)
          int any = 0, bad = 0;
          const double adj = sqrt(cabs2(dj));
          for (int v = lane; v < nv; v += 32) {
            if (!s_act[v]) continue;
            const double tw = s_tot[v][0], tp = s_tot[v][1];
            const double ej = adj * sqrt(tw), pn = sqrt(tp);
            if (!isfinite(ej) || !isfinite(pn)) bad = 1;
            if (ej + s_ep[v] <= a.tol_abs + a.tol_rel * pn) {
              s_act[v] = 0;
              s_m[v] = j;
              s_pn[v] = pn;
            } else {
              s_ep[v] = ej;
              any = 1;
            }
          }
          any = __any_sync(kFull, any);
          bad = __any_sync(kFull, bad);
          if (lane == 0) s_flag = bad ? 2 : (any ? 0 : 1);
        }
        __syncthreads();
        it++;
        if (s_flag == 2) { fail(MAGNUS_ENONFINITE); return; }
        if (s_flag == 1) {
          // nothing reads the gathered maxima of this iteration: clear them for the next substep
          if (TC && b == 0)
            for (int c = tid; c < kTcCols; c += blockDim.x) a.colmax[3 * kTcCols + c] = 0ull;
          done = true;
          break;
        }
        if (TC && j < a.m_max) {  // digits of w_j from the maxima gathered in the epilogue
          const int set = ((j - 1) & 1) ? 2 : 1;
          const unsigned long long *cm = a.colmax + 3 * kTcCols;
          int *exps = tc_set_exps(set);
          for (int c = tid; c < 2 * nv; c += blockDim.x) {
            s_cexp[c] = cover_exponent(__longlong_as_double((long long)cm[c]));
            if (b == 0) exps[c] = s_cexp[c];
          }
          __syncthreads();
          __nv_bfloat16 *dg = (__nv_bfloat16 *)tc_set_digits(set);
          const int ncol = 2 * nv;
          const int64_t ngroups = (hi - lo) / 8;
          for (int64_t w = tid; w < ngroups * ncol; w += blockDim.x) {
            const int c = (int)(w % ncol), v = c >> 1;
            const int64_t r0 = lo + 8 * (w / ncol);
            double xv[8];
#pragma unroll
            for (int i = 0; i < 8; i++) {
              const double2 x = dst[(int64_t)v * D + r0 + i];
              // a vector that stopped keeps its old w: its products are not used, its digits are 0
              xv[i] = s_act[v] ? ((c & 1) ? x.y : x.x) : 0.0;
            }
            tcg::slice8_tiled(xv, s_cexp[c], dg, D, c, r0);
          }
          asm volatile("fence.proxy.async.global;" ::: "memory");
          if (!grid_barrier(a.bar, G, a.spin_limit_ns)) { fail(MAGNUS_ETIMEOUT); return; }
          // every block has read the gathered maxima: block 0 clears them before its next barrier
          if (b == 0)
            for (int c = tid; c < kTcCols; c += blockDim.x) a.colmax[3 * kTcCols + c] = 0ull;
        }
      }
      if (!done) { fail(MAGNUS_ENOCONV); return; }
      if (tid == 0) {  // a posteriori norm check of the substep (every block decides alike)
        int bad = 0;
        for (int v = 0; v < nv; v++)
          bad |= drift_fails(s_pn[v], s_vn[v], a.tol_abs, a.tol_rel, a.norm_check, a.counters, b == 0) ? 1 : 0;
        s_drift = bad;
      }
      __syncthreads();
      if (s_drift) { fail(MAGNUS_EDRIFT); return; }
      if (tid < nv) s_vn[tid] = s_pn[tid];
      if (b == 0 && tid == 0) {
        Counters *c = a.counters;
        for (int v = 0; v < nv; v++) {
          const int m = s_m[v];
          c->n_matvec += m;
          c->n_termapply += (long long)m * nt * (R.mode == MODE_M4 ? 2 : 1);
          if (m > c->max_m) c->max_m = m;
          if (a.mlog && sub_counter * nv + v < a.mlog_cap) a.mlog[sub_counter * nv + v] = m;
        }
        c->n_substeps += nv;
      }
      __syncthreads();
      sub_counter++;
      double2 *tmp = cur; cur = nxt; nxt = tmp;
    }
    if (b == 0 && tid == 0) a.counters->n_exp++;
  }
  if (cur != a.psi)
    for (int v = 0; v < nv; v++)
      for (int64_t r = lo + tid; r < hi; r += blockDim.x) a.psi[(int64_t)v * D + r] = cur[(int64_t)v * D + r];
}

const void *dense_kernel(bool real, bool tiled, int prec) {
  if (prec == 1) return (const void *)k_dense_persistent<true, true, 1>;
  if (prec == 3) return (const void *)k_dense_persistent<true, true, 3>;
  if (prec == 4) return (const void *)k_dense_persistent<true, true, 4>;
  if (real)
    return tiled ? (const void *)k_dense_persistent<true, true, 0> : (const void *)k_dense_persistent<true, false, 0>;
  return tiled ? (const void *)k_dense_persistent<false, true, 0> : (const void *)k_dense_persistent<false, false, 0>;
}

cudaError_t tc_smem_attr() {
  static bool done = false;
  if (done) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(dense_kernel(true, true, 3), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)tcg::kSmemBytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(dense_kernel(true, true, 4), cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)tcg::kSmemBytes);
  if (e == cudaSuccess) done = true;
  return e;
}

size_t dyn_smem(int prec) { return prec >= 3 ? tcg::kSmemBytes : 0; }

}  // namespace

int dense_block_size() { return kDBlock; }
int dense_rows_per_unit(bool tiled) { return tiled ? kTM : 1; }

namespace {
__global__ void k_split_dense(const double *Hr, int rs, float2 *out, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double x = Hr[i * rs];
    const float hi = __double2float_rn(x);
    out[i] = make_float2(hi, __double2float_rn(x - (double)hi));
  }
}
}  // namespace


namespace {
// one warp per row: row maximum -> exponent, then the row's 4 digits of 8 bits
__global__ void k_slice_dense_tc(const double *Hr, int rs, int64_t D, __nv_bfloat16 *digits, int *rexp) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < D; r += nw) {
    double m = 0.0;
    for (int64_t c = lane; c < D; c += 32) m = fmax(m, fabs(Hr[(r * D + c) * rs]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(kFull, m, o));
    const int e = tcg::cover_exponent(m);
    if (lane == 0) rexp[r] = e;
    for (int64_t c = lane; c < D; c += 32) tcg::slice_value_tiled(Hr[(r * D + c) * rs], e, digits, D, r, c);
  }
}
}  // namespace

cudaError_t launch_slice_dense_tc(const double *Hr, int rs, int64_t D, void *digits, int *rexp, cudaStream_t st) {
  k_slice_dense_tc<<<152 * 8, 256, 0, st>>>(Hr, rs, D, (__nv_bfloat16 *)digits, rexp);
  return cudaGetLastError();
}

size_t dense_tc_smem_bytes() { return tcg::kSmemBytes; }

int dense_tc_chunk(int64_t D) { return tcg::chunk_for(D); }

int dense_tc_slots(int ndense, int64_t D, int grid) {
  const long long T = D / tcg::kM, C = D / tcg::chunk_for(D);
  const long long N = (long long)ndense * T * C;
  int slots = 1;
  for (int b = 0; b < grid; b++) {
    const long long i0 = tcg::range_lo(b, grid, N), i1 = tcg::range_lo(b + 1, grid, N);
    if (i0 < i1) slots = std::max(slots, (int)((i1 - 1) / C - i0 / C + 1));
  }
  return slots;
}

cudaError_t launch_split_dense(const double *Hr, int rs, float2 *out, int64_t n, cudaStream_t st) {
  k_split_dense<<<152 * 8, 256, 0, st>>>(Hr, rs, out, n);
  return cudaGetLastError();
}

cudaError_t dense_max_blocks_per_sm(int *n) {
  int best = 1 << 30;
  cudaError_t e0 = tc_smem_attr();
  if (e0 != cudaSuccess) return e0;
  for (int r = 0; r < 2; r++)
    for (int t = 0; t < 5; t++) {
      int k = 0;
      const int prec = t < 2 ? 0 : (t == 2 ? 1 : t);  // FP64 warp rows, FP64 tiles, split, tcgen05, tcgen05 M4
      cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&k, dense_kernel(r, t > 0, prec), kDBlock,
                                                                    dyn_smem(prec));
      if (e != cudaSuccess) return e;
      best = k < best ? k : best;
    }
  *n = best;
  return cudaSuccess;
}

cudaError_t launch_dense_persistent(const PersistArgs &a, bool real_valued, int grid, cudaStream_t st) {
  PersistArgs copy = a;
  void *args[] = {&copy};
  const int prec = a.tc ? 2 + a.tc : (a.split ? 1 : 0);
  if (prec >= 3) {
    cudaError_t e = tc_smem_attr();
    if (e != cudaSuccess) return e;
  }
  return cudaLaunchCooperativeKernel(dense_kernel(real_valued, a.nvec > 1 || prec > 0, prec), dim3(grid),
                                     dim3(kDBlock), args, dyn_smem(prec), st);
}

}  // namespace mg
