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
// Per-vector stop decisions: each block writes its per-vector partial sums; after a barrier, block
// v sums vector v's partials over all blocks in a fixed order; after a second barrier every block
// reads the same totals and takes the same decisions.
#include <math.h>

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
__device__ __forceinline__ void gemm_tile(DenseSmem &S, const double2 *H, double coef, const double2 *W, int64_t D,
                                          int nv, int64_t r0, int64_t rend, double2 (&acc)[2][4]) {
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  for (int64_t k0 = 0; k0 < D; k0 += kTK) {
    __syncthreads();
    // stage coef * H[r0 .. r0+31][k0 .. k0+31] (coalesced along the row)
    for (int i = tid; i < kTM * kTK; i += kDBlock) {
      const int rr = i / kTK, kk = i % kTK;
      const int64_t row = r0 + rr, col = k0 + kk;
      double2 v = make_double2(0.0, 0.0);
      if (row < rend && col < D) v = __ldg(H + row * D + col);
      S.h[rr][kk] = coef * v.x;
      if (!REAL) S.hi[rr][kk] = coef * v.y;
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
__device__ __forceinline__ double2 gemv_row_partial(const double2 *H, const double2 *x, int64_t D, int64_t r) {
  const int lane = threadIdx.x & 31;
  double2 acc = make_double2(0.0, 0.0);
  const double2 *row = H + r * D;
  int64_t j = lane;
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

// ------------------------------------------------------------------ kernel
template <bool REAL, bool TILED, bool SPLIT>
__global__ void __launch_bounds__(kDBlock, 1) k_dense_persistent(PersistArgs a) {
  __shared__ Term sT[kMaxTerms];
  __shared__ ExpRec sR;
  __shared__ double s_vn[kVecMax], s_ep[kVecMax], s_pn[kVecMax];
  __shared__ int s_act[kVecMax], s_m[kVecMax];
  __shared__ double s_part[kDBlock / 32][kVecMax][2];
  __shared__ int s_flag;
  __shared__ TileSmem TS;
  DenseSmem &S = TS.d;

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

  double *partials = a.partials;                        // [2][G][nv][2]
  double *totals = a.partials + (size_t)4 * G * nv;     // [2][nv][2]
  unsigned it = 0;
  auto fail = [&](int status) {
    if (tid == 0) atomicCAS(&a.counters->status, 0, status);
  };

  // Reduce per-thread per-vector sums (tiled: vectors tx + 16 q; warp-per-row: the lane's own
  // vector 0) to this block's partials, barrier, per-vector totals by block v, barrier.
  auto reduce_and_share = [&](double (&sw)[4], double (&sp)[4]) -> bool {
    double *slot = partials + (size_t)(it & 1u) * G * nv * 2;
    if (TILED) {
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
    if (warp == 0)
      for (int v = b; v < nv; v += G) {  // block b sums the vectors v = b, b + G, ...
        double y0 = 0.0, y1 = 0.0;
        for (int q = lane; q < (int)G; q += 32) {
          y0 += slot[((size_t)q * nv + v) * 2];
          y1 += slot[((size_t)q * nv + v) * 2 + 1];
        }
        y0 = warp_sum(y0);
        y1 = warp_sum(y1);
        if (lane == 0) {
          totals[((it & 1u) * nv + v) * 2] = y0;
          totals[((it & 1u) * nv + v) * 2 + 1] = y1;
        }
      }
    return grid_barrier(a.bar, G, a.spin_limit_ns);
  };

  // y[i][q] = sum_k coef_k (H_k src)[row][vec] (+ field), for this thread's outputs
  // tiled: rows r0 + 2 ty + i, vectors tx + 16 q.  warp path: row r, vector 0 (lane 0 holds it).
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
          if (SPLIT)
            gemm_tile_split(TS.f, a.hsplit[k], coef[k], shs[k], D, nv, r0, hi, y);
          else
            gemm_tile<REAL>(S, sT[k].val, coef[k], srcs[k], D, nv, r0, hi, y);
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
          const double2 part = gemv_row_partial<REAL>(sT[k].val, srcs[k], D, r0);
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
    if (tid < nv) s_vn[tid] = sqrt(totals[((it & 1u) * nv + tid) * 2]);
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
        if (R.mode == MODE_M4) {
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
        }
        double sw[4] = {0, 0, 0, 0}, sp[4] = {0, 0, 0, 0};
        // epilogue for one output (row r, vector v) with y = the combined matvec
        auto finish = [&](int64_t r, int v, double2 y, int q) {
          const int64_t idx = (int64_t)v * D + r;
          const double2 wr = ldv(src + idx);
          y = rfma(-shift, wr, y);
          dst[idx] = y;
          if (SPLIT) dst_sh[idx] = split4(y);
          double2 pr = (j == 1) ? cmul(d0, wr) : nxt[idx];
          pr = cfma(dj, y, pr);
          nxt[idx] = pr;
          sw[q] += cabs2(y);
          sp[q] += cabs2(pr);
        };
        auto commutator = [&](int64_t r0, double2 (&y)[2][4]) {
          // y += sum_k bg_k u_k - i sum_{k<l} kg_kl (H_k u_l - H_l u_k)
          int pi = 0;
          for (int k = 0; k < nt; k++)
            for (int l = k + 1; l < nt; l++, pi++) {
              if (R.kg[pi] == 0.0) continue;
              double ck[kMaxTerms] = {0, 0, 0, 0}, cl[kMaxTerms] = {0, 0, 0, 0};
              ck[k] = R.kg[pi];
              cl[l] = -R.kg[pi];
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
            }
        };
        if (TILED) {
          for (int64_t r0 = lo; r0 < hi; r0 += kTM) {
            double2 y[2][4];
            if (R.mode == MODE_M4) {
              for (int i = 0; i < 2; i++)
                for (int q = 0; q < 4; q++) y[i][q] = make_double2(0.0, 0.0);
              commutator(r0, y);
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
        if (!reduce_and_share(sw, sp)) { fail(MAGNUS_ETIMEOUT); return; }
        if (warp == 0) {
          int any = 0, bad = 0;
          const double adj = sqrt(cabs2(dj));
          if (lane == 0)
            for (int v = 0; v < nv; v++) {
              if (!s_act[v]) continue;
              const double tw = totals[((it & 1u) * nv + v) * 2], tp = totals[((it & 1u) * nv + v) * 2 + 1];
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
          if (lane == 0) s_flag = bad ? 2 : (any ? 0 : 1);
        }
        __syncthreads();
        it++;
        if (s_flag == 2) { fail(MAGNUS_ENONFINITE); return; }
        if (s_flag == 1) { done = true; break; }
      }
      if (!done) { fail(MAGNUS_ENOCONV); return; }
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

const void *dense_kernel(bool real, bool tiled, bool split) {
  if (split) return (const void *)k_dense_persistent<true, true, true>;
  if (real)
    return tiled ? (const void *)k_dense_persistent<true, true, false> : (const void *)k_dense_persistent<true, false, false>;
  return tiled ? (const void *)k_dense_persistent<false, true, false> : (const void *)k_dense_persistent<false, false, false>;
}

}  // namespace

int dense_block_size() { return kDBlock; }
int dense_rows_per_unit(bool tiled) { return tiled ? kTM : 1; }

namespace {
__global__ void k_split_dense(const double2 *H, float2 *out, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double x = H[i].x;
    const float hi = __double2float_rn(x);
    out[i] = make_float2(hi, __double2float_rn(x - (double)hi));
  }
}
}  // namespace

cudaError_t launch_split_dense(const double2 *H, float2 *out, int64_t n, cudaStream_t st) {
  k_split_dense<<<152 * 8, 256, 0, st>>>(H, out, n);
  return cudaGetLastError();
}

cudaError_t dense_max_blocks_per_sm(int *n) {
  int best = 1 << 30;
  for (int r = 0; r < 2; r++)
    for (int t = 0; t < 3; t++) {
      int k = 0;
      cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&k, dense_kernel(r, t > 0, t == 2), kDBlock, 0);
      if (e != cudaSuccess) return e;
      best = k < best ? k : best;
    }
  *n = best;
  return cudaSuccess;
}

cudaError_t launch_dense_persistent(const PersistArgs &a, bool real_valued, int grid, cudaStream_t st) {
  PersistArgs copy = a;
  void *args[] = {&copy};
  return cudaLaunchCooperativeKernel(dense_kernel(real_valued, a.nvec > 1 || a.split, a.split != 0), dim3(grid),
                                     dim3(kDBlock), args, 0, st);
}

}  // namespace mg
