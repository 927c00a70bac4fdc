// Exact-digit dense products on the 5th-generation tensor cores (MAGNUS_TENSOR_SLICED).
// Y_k = H_k W_k for every dense term k and a set W_k of up to 128 real columns (the real and
// imaginary parts of up to 64 states; one set for all terms in the linear generators, the set of
// u_l for term k in the commutators of M4), with H_k and W_k given as 4 signed 8-bit digits per value:
//     H[r][j] = 2^{e_r} sum_t h_t[r][j] 2^{-8(t+1) + 1},   W[c][j] = 2^{e_c} sum_u w_u[c][j] 2^{-8(u+1) + 1},
// (a value scaled to 31 bits, N = round(x 2^{31-e}), cut into balanced base-256 digits) with every
// |h_t|, |w_u| <= 128, all exact in bf16.  The digit products of level g = t + u <= 3 (10 of the 16
// pairs) are summed by tcgen05.mma (kind::f16) into four FP32 accumulators in tensor memory, one
// 128 x 128 tile each (all 512 TMEM columns):
//   * levels 0 and 1 restart every chunk of 512 K values (the largest of 512, 256, 128 dividing D);
//     per K index |h_0 w_0| <= 2^14 and |h_0 w_1 + h_1 w_0| <= 2^15, so every partial sum is an
//     integer of magnitude at most 2^24, which FP32 holds exactly; the chunk sums are moved to
//     int64 (S = 2^8 L_0 + L_1) after each chunk;
//   * levels 2 and 3 (weights 2^-16 and 2^-24 of level 0) accumulate in FP32 over the whole range;
//     their rounding is below 2^-40 of the product scale.
// The value is Y[r][c] = 2^{e_r + e_c - 22} (S + (L_2 + L_3 2^-8) 2^-8).  The truncation after four
// digits and the omitted levels 4..6 leave below D * 2^-29 * max_j |H_rj| * max_j |W_cj| per entry.
//
// Work split: the items (dense term, 128-row tile, K chunk) in that order are cut into G contiguous
// ranges, one per CTA; a CTA accumulates consecutive chunks of the same tile and writes one FP64
// partial tile per (tile it touched) into its own slots; the caller sums the partials of a tile in
// CTA order after a grid barrier (deterministic).
//
// Layout: the digits live in global memory already in the order the MMA reads them from shared
// memory (K-major, no swizzle, core matrices of 8 rows x 16 B): a block of 8 K values is
// [4 digits][128 rows][8] bf16 = 8 KB, and the blocks of consecutive K follow each other, so
//   H digits: [term][row tile][D / 8 K-blocks][4][128][8],   vector digits: [set][D / 8][4][128][8]
// and one pipeline stage (32 K) of either operand is one contiguous 32 KB bulk copy (TMA bulk
// engine, cp.async.bulk) into a 3-deep ring of 64 KB stages.  One thread issues the copies and the
// MMAs; all 8 warps move the accumulators out of tensor memory.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

#include "tcgen05.cuh"

namespace mg {
namespace tcg {

constexpr int kSl = 4;                          // digits per value
constexpr int kM = 128;                         // rows per tile (MMA M)
constexpr int kN = 128;                         // columns (MMA N)
constexpr int kKS = 32;                         // K per pipeline stage
constexpr int kChunkMax = 512;                  // K per exact chunk (512, or the largest of 256, 128 dividing D)
constexpr int kNBits = 31;                      // values scaled to kNBits bits before cutting into digits
constexpr int kNS = 3;                          // ring depth
constexpr uint32_t kBox = 8 * kM * kSl * 2;     // 8 KB: one TMA box (8 K x 128 rows x 4 digits)
constexpr uint32_t kStageA = 4 * kBox;          // 32 KB: the 4 K-cores of a stage
constexpr uint32_t kStageBytes = 2 * kStageA;   // A and B
constexpr size_t kSmemBytes = (size_t)kNS * kStageBytes + 1024;  // + alignment slack
constexpr uint32_t kTmemCols = 512;             // 4 levels x 128 columns
constexpr uint32_t kIdesc = tc::idesc_bf16(kM, kN);
constexpr uint32_t kIdesc2 = tc::idesc_bf16(kM, 2 * kN);  // two adjacent levels at once
constexpr int kThreads = 256;                   // 8 warps: lane quadrant = warp % 4, column half = warp / 4

struct Bars {
  uint64_t full[kNS];
  uint64_t empty[kNS];
  uint64_t accr;
  uint32_t tmem;
  uint32_t _pad;
};

// running counters of the ring and of the chunk barrier; identical in every thread of the CTA
struct Pipe {
  uint32_t stage;  // stages issued so far
  uint32_t chunk;  // chunks completed so far
};

// the vector set each dense term multiplies in one product phase (its digits and column exponents):
// the same set for every term in the linear generators; in the commutator phases of M4, term k
// multiplies the set of u_l
constexpr int kMaxSets = 4;
struct Sets {
  const __nv_bfloat16 *wd[kMaxSets];
  const int *ec[kMaxSets];
};

struct Geometry {
  int ndense;       // dense terms
  int T;            // row tiles (D / 128)
  int C;            // chunks per tile (D / chunk)
  int chunk;        // K per chunk (256 or 128)
  long long N;      // items = ndense * T * C
  int slots;        // partial tiles per CTA
};

// first item of CTA b's range (32-bit division when the product fits, the common case)
__host__ __device__ inline long long range_lo(long long b, int G, long long N) {
  const long long p = b * N;
  return p < 2147483647ll ? (long long)((unsigned)p / (unsigned)G) : p / G;
}

// element offset of digit t of element (row r, K index j) in the tiled layout with K extent D
__host__ __device__ inline size_t tiled_offset(int64_t D, int64_t r, int64_t j, int t) {
  return ((((size_t)(r / kM) * (size_t)(D / 8) + (size_t)(j / 8)) * kSl + t) * kM + (size_t)(r % kM)) * 8 + (size_t)(j % 8);
}

// K per exact chunk for dimension D (a multiple of 128)
__host__ __device__ inline int chunk_for(int64_t D) { return D % 512 == 0 ? 512 : (D % 256 == 0 ? 256 : 128); }

// x (finite, |x| < 2^e) -> N = round(x 2^{31 - e}), |N| <= 2^31, from the bits of x (integer pipe
// only: on this part the FP64 pipe is the scarce one)
__device__ __forceinline__ long long fixed32(double x, int e) {
  const long long bits = __double_as_longlong(x);
  const int ex = (int)((bits >> 52) & 0x7FF);
  if (ex == 0) return 0;                            // zero (or subnormal: below 2^-1022 <= 2^{e-31} here)
  const long long mant = (bits & 0xFFFFFFFFFFFFFll) | 0x10000000000000ll;
  const int sh = e + 1075 - kNBits - ex;            // x 2^{31-e} = mant 2^{-sh}; sh >= 22 as |x| < 2^e
  long long n = sh >= 63 ? 0 : ((mant >> (sh - 1)) + 1) >> 1;  // round half up in magnitude
  return bits < 0 ? -n : n;
}

// N -> 4 balanced base-256 digits d_t (N = sum_t d_t 2^{8(3-t)}, every |d_t| <= 128 for |N| <= 2^31)
__device__ __forceinline__ void digits4(long long n, int (&d)[kSl]) {
  d[0] = (int)((n + (1ll << 23)) >> 24);
  n -= (long long)d[0] << 24;
  d[1] = (int)((n + (1ll << 15)) >> 16);
  n -= (long long)d[1] << 16;
  d[2] = (int)((n + (1ll << 7)) >> 8);
  d[3] = (int)(n - ((long long)d[2] << 8));
}

// one value -> 4 digits of 8 bits with exponent e (|x| < 2^e), written to the tiled layout
// (row r = tile row or vector column, K index j): x 2^-e = sum_t d_t 2^{-8(t+1)} + O(2^-33)
__device__ __forceinline__ void slice_value_tiled(double x, int e, __nv_bfloat16 *base, int64_t D, int64_t r, int64_t j) {
  int d[kSl];
  digits4(fixed32(x, e), d);
#pragma unroll
  for (int t = 0; t < kSl; t++) base[tiled_offset(D, r, j, t)] = __int2bfloat16_rn(d[t]);
}

// digits of 8 consecutive K values (j0 % 8 == 0) of one row/column r, packed: four 16-byte stores
// into the tiled layout (digit t of the 8 values is one 16-byte piece)
__device__ __forceinline__ void slice8_tiled(const double (&x)[8], int e, __nv_bfloat16 *base, int64_t D, int64_t r,
                                             int64_t j0) {
  uint32_t packed[kSl][4];
#pragma unroll
  for (int i = 0; i < 8; i += 2) {
    int d0[kSl], d1[kSl];
    digits4(fixed32(x[i], e), d0);
    digits4(fixed32(x[i + 1], e), d1);
#pragma unroll
    for (int t = 0; t < kSl; t++) {
      const uint32_t lo = __bfloat16_as_ushort(__int2bfloat16_rn(d0[t]));
      const uint32_t hi = __bfloat16_as_ushort(__int2bfloat16_rn(d1[t]));
      packed[t][i / 2] = lo | (hi << 16);
    }
  }
#pragma unroll
  for (int t = 0; t < kSl; t++)
    *reinterpret_cast<uint4 *>(base + tiled_offset(D, r, j0, t)) =
        make_uint4(packed[t][0], packed[t][1], packed[t][2], packed[t][3]);
}

__device__ __forceinline__ int cover_exponent(double m) {
  int e = 0;
  if (m > 0.0) frexp(m, &e);
  return e;
}

// Y_k = H_k W_k for every dense term k, W_k given by W.wd[k] (tiled digits) and W.ec[k] (its column
// exponents [kN]), this CTA's range.  hd: tiled digits of all dense terms; P: partial tiles
// [G][slots][kN cols][kM rows] (FP64, column-major in the tile); eh: row exponents [ndense][D].
// smem: kSmemBytes of dynamic shared memory.  Returns false if a bounded wait ran out (the caller
// reports MAGNUS_ETIMEOUT).
__device__ bool gemm_phase(const __nv_bfloat16 *hd, const Sets &W, const Geometry &g, const int *eh, double *P,
                           unsigned char *smem_raw, Bars &bars, Pipe &pipe, long long max_spins) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int b = blockIdx.x, G = gridDim.x;
  unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const long long i0 = range_lo(b, G, g.N), i1 = range_lo(b + 1, G, g.N);
  const long long D = (long long)g.T * kM;
  if (i0 >= i1) return true;

  if (warp == 0) tc::tmem_alloc(&bars.tmem, kTmemCols);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = bars.tmem;
  bool ok = true;

  const int quad = warp & 3, half = warp >> 2;
  const int row = quad * 32 + lane;           // TMEM lane = tile row
  const uint32_t lane_base = (uint32_t)(quad * 32) << 16;
  long long S[kN / 2];                        // exact levels 0, 1 of this thread's 64 columns

  const int spc = g.chunk / kKS;  // stages per chunk
  const long long nstages = (i1 - i0) * spc;
  // stage j of the range -> item i0 + j / 4, K offset
  auto load_stage = [&](long long j) {
    const uint32_t gs = pipe.stage + (uint32_t)j;
    const int buf = (int)(gs % kNS);
    const long long item = i0 + j / spc;
    const long long tile = item / g.C;
    const long long k0 = (item % g.C) * g.chunk + (j % spc) * kKS;
    unsigned char *sa = smem + (size_t)buf * kStageBytes, *sb = sa + kStageA;
    // tile = term * T + row tile: its K-blocks start at tile * (D / 8) blocks of kBox bytes
    const unsigned char *ga = (const unsigned char *)hd + ((size_t)tile * (size_t)(D / 8) + (size_t)(k0 / 8)) * kBox;
    const unsigned char *gb = (const unsigned char *)W.wd[(int)(tile / g.T)] + (size_t)(k0 / 8) * kBox;
    tc::mbar_expect_tx(&bars.full[buf], kStageBytes);
    tc::bulk_load(sa, ga, kStageA, &bars.full[buf]);
    tc::bulk_load(sb, gb, kStageA, &bars.full[buf]);
  };

  // the issuing thread: prologue loads (after making the generic-proxy writes of the digits visible)
  if (tid == 0) {
    asm volatile("fence.proxy.async.global;" ::: "memory");
    for (long long j = 0; j < nstages && j < kNS; j++) {
      const uint32_t gs = pipe.stage + (uint32_t)j;
      if (gs >= kNS && !tc::mbar_wait(&bars.empty[gs % kNS], ((gs / kNS) - 1) & 1u, max_spins)) ok = false;
      if (ok) load_stage(j);
    }
  }

  const uint64_t desc0 = tc::smem_desc(tc::smem_u32(smem), kBox, 128);  // buffer 0, K-block 0, digit 0
  long long j = 0;        // next stage to issue
  int slot = 0;
  for (long long item = i0; item < i1; item++) {
    const long long tile = item / g.C;
    const bool tile_start = (item == i0) || (item % g.C == 0);
    const bool tile_end = (item + 1 == i1) || ((item + 1) % g.C == 0);
    if (tile_start) {
#pragma unroll
      for (int q = 0; q < kN / 2; q++) S[q] = 0;
    }
    // ---- issue the chunk's 4 stages (one thread)
    if (tid == 0) {
      for (int st = 0; st < spc && ok; st++, j++) {
        const uint32_t gs = pipe.stage + (uint32_t)j;
        const int buf = (int)(gs % kNS);
        if (!tc::mbar_wait(&bars.full[buf], (gs / kNS) & 1u, max_spins)) { ok = false; break; }
        tc::fence_after_sync();
        // descriptors differ only in their start-address field (address / 16, 14 bits: every
        // shared-memory address fits), so each is the stage's base descriptor plus a constant
        const uint64_t abase = desc0 + ((uint64_t)(buf * kStageBytes) >> 4);
        const uint64_t bbase = abase + (kStageA >> 4);
        const uint32_t reset = (st == 0 ? 0x3u : 0u) | ((st == 0 && tile_start) ? 0xCu : 0u);
#pragma unroll
        for (int ks = 0; ks < kKS / 16; ks++) {
          // digit t of H against the pair of vector digits (u, u + 1), stacked as one 256-row
          // operand (digit planes are 2 KB apart, so the pair is contiguous), writes the adjacent
          // accumulators of levels t + u and t + u + 1 in one N = 256 product; the last pair of
          // rows t = 1 and t = 3 has a single digit left (N = 128)
          const uint32_t ko = (uint32_t)(2 * ks) * kBox;
#pragma unroll
          for (int t = 0; t < kSl; t++)
#pragma unroll
            for (int u = 0; u + t <= 3; u += 2) {
              const int lvl = t + u;
              const bool pair = (lvl + 1 <= 3);
              const uint64_t ad = abase + ((ko + (uint32_t)t * 2048u) >> 4);
              const uint64_t bd = bbase + ((ko + (uint32_t)u * 2048u) >> 4);
              // t = 0 opens every level (levels 0, 1 together, 2, 3 together) in the first K step of a
              // stage where they restart (levels 0, 1 every chunk, 2, 3 every tile)
              const uint32_t acc = (ks == 0 && t == 0 && ((reset >> lvl) & 1u)) ? 0u : 1u;
              tc::mma_bf16(tmem + (uint32_t)lvl * kN, ad, bd, pair ? kIdesc2 : kIdesc, acc);
            }
        }
        tc::mma_commit(&bars.empty[buf]);
        // refill the buffer of the previous stage once its MMAs are done
        if (j >= 1 && j - 1 + kNS < nstages) {
          const uint32_t gp = pipe.stage + (uint32_t)(j - 1);
          if (!tc::mbar_wait(&bars.empty[gp % kNS], (gp / kNS) & 1u, max_spins)) { ok = false; break; }
          load_stage(j - 1 + kNS);
        }
      }
      tc::mma_commit(&bars.accr);
    }
    __syncwarp();
    // ---- chunk accumulators -> int64 (all warps); a failed wait anywhere stops the whole CTA
    const bool got = tc::mbar_wait(&bars.accr, pipe.chunk & 1u, max_spins);
    pipe.chunk++;
    ok = __syncthreads_and((ok && got) ? 1 : 0) != 0;
    tc::fence_after_sync();
    if (ok) {
#pragma unroll
      for (int c16 = 0; c16 < 4; c16++) {
        uint32_t v0[16], v1[16];
        const uint32_t col = (uint32_t)(half * 64 + c16 * 16);
        tc::tmem_ld16(tmem + lane_base + 0 * kN + col, v0);
        tc::tmem_ld16(tmem + lane_base + 1 * kN + col, v1);
        tc::tmem_ld_wait();
#pragma unroll
        for (int q = 0; q < 16; q++)
          S[c16 * 16 + q] += ((long long)__float2int_rn(__uint_as_float(v0[q])) << 8) +
                             (long long)__float2int_rn(__uint_as_float(v1[q]));
      }
    }
    if (ok && tile_end) {
      // FP64 partial tile: levels 0/1 exact, 2/3 from tensor memory
      const int term = (int)(tile / g.T), r0 = (int)(tile % g.T) * kM;
      const int er = eh[(long long)term * D + r0 + row];
      const int *ec = W.ec[term];
      double *out = P + ((size_t)b * g.slots + slot) * (size_t)(kN * kM);
#pragma unroll
      for (int c16 = 0; c16 < 4; c16++) {
        uint32_t v2[16], v3[16];
        const uint32_t col = (uint32_t)(half * 64 + c16 * 16);
        tc::tmem_ld16(tmem + lane_base + 2 * kN + col, v2);
        tc::tmem_ld16(tmem + lane_base + 3 * kN + col, v3);
        tc::tmem_ld_wait();
#pragma unroll
        for (int q = 0; q < 16; q++) {
          const int cc = (int)col + q;
          const double lo = ((double)__uint_as_float(v2[q]) + (double)__uint_as_float(v3[q]) * 0x1.0p-8) * 0x1.0p-8;
          // 2^{e_r + e_c - 2 kNBits + 40} (= 2^{e_r + e_c - 22}) from its exponent bits when it is normal
          const int bx = er + ec[cc] - 2 * kNBits + 40 + 1023;
          const double sc = (bx > 0 && bx < 2047) ? __longlong_as_double((long long)bx << 52) : ldexp(1.0, bx - 1023);
          out[(size_t)cc * kM + row] = fma((double)S[c16 * 16 + q], sc, lo * sc);
        }
      }
      slot++;
    }
    tc::fence_before_sync();
    __syncthreads();  // tensor memory free for the next chunk's (or tile's) restarting levels
    tc::fence_after_sync();
    if (!ok) break;
  }
  pipe.stage += (uint32_t)nstages;
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, kTmemCols);
  return ok;
}

// The CTAs whose ranges hold the chunks of tile `tile` (global tile index term * T + r), and for
// each its slot; the caller sums P over them in this order.
__host__ __device__ inline void tile_owners(long long tile, const Geometry &g, int G, int *b_first, int *b_last) {
  const long long t0 = tile * g.C, t1 = t0 + g.C;  // items [t0, t1)
  *b_first = (int)(((t0 + 1) * G - 1) / g.N);
  *b_last = (int)((t1 * G - 1) / g.N);
}
__host__ __device__ inline int tile_slot(long long tile, int b, const Geometry &g, int G) {
  return (int)(tile - range_lo(b, G, g.N) / g.C);
}

}  // namespace tcg
}  // namespace mg
