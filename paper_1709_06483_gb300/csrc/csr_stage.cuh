// Staged CSR rows for the fixed-point Leja pass (FAM_CSR, linear generators): each warp takes the
// block's rows in tiles of 32 (one row per lane) and reads the matrix of a tile from shared memory.
// A tile's rows own one contiguous run of every term's arrays -- columns, and for product terms
// the 62-bit value mantissas -- so one lane copies those runs into a slot of the warp's shared
// memory with cp.async.bulk (the TMA bulk engine) two tiles ahead of the one the warp computes,
// completion counted on the slot's mbarrier.  The lanes then walk their rows in shared memory and
// only the gathers of the fixed-point vector go to global memory.  The matrix is the same in every
// Leja iteration, so the pipeline runs on across iterations: the copies issued at the end of a pass
// are the first tiles of the next one.
//
// Sums and products are exact 64-bit integers (rows.cuh), so the order in which a row's entries are
// read does not change the result: a staged row gives the bits the unstaged row gives.  A tile
// whose runs do not fit a slot, or would reach past the last 16-byte block of an array, is read
// from global memory by the unstaged rows (its copy is an empty arrival).
#pragma once

#include "rows.cuh"
#include "tcgen05.cuh"

namespace mg {
namespace stage {

constexpr int kWarps = 8;            // warps per CTA (256 threads)
constexpr int kTile = 32;            // rows per tile, one per lane
constexpr int kSlotBytes = 9472;     // one slot; 74 x 128 B (the 20-spin chain's largest tile needs 9328)
constexpr size_t kSmemBytes = (size_t)kWarps * 2 * kSlotBytes;  // 151,552 B of dynamic shared memory
constexpr int kRound = 16;           // gathers in flight per lane

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Byte runs of one tile inside a slot: run 2k holds term k's columns, run 2k+1 its mantissas.
struct Lay {
  uint32_t off[2 * kMaxTerms];  // offset of the run in the slot
  int64_t b0[2 * kMaxTerms];    // first byte of the run in the global array (16-byte aligned)
  uint32_t len[2 * kMaxTerms];  // bytes (a multiple of 16, possibly 0)
  uint32_t total;
  bool fits;
};

// entry range [e0, e1) of term t over rows [ra, rb): row pointers, or r * plen for rows of one length
__device__ __forceinline__ void term_span(const Term &t, int64_t ra, int64_t rb, int64_t &e0, int64_t &e1) {
  if (t.plen) {
    e0 = ra * t.plen;
    e1 = rb * t.plen;
  } else {
    e0 = __ldg(t.rowptr + ra);
    e1 = __ldg(t.rowptr + rb);
  }
}

__device__ __forceinline__ void layout(const Term *T, int nt, const int64_t (&e0)[kMaxTerms],
                                       const int64_t (&e1)[kMaxTerms], Lay &L) {
  uint32_t off = 0;
  bool fits = true;
#pragma unroll
  for (int k = 0; k < kMaxTerms; k++) {
#pragma unroll
    for (int v = 0; v < 2; v++) {
      const int q = 2 * k + v;
      L.off[q] = off;
      L.b0[q] = 0;
      L.len[q] = 0;
      if (k >= nt || (v == 1 && T[k].pattern)) continue;
      const int es = v ? 8 : 4;  // bytes per entry
      const int64_t b0 = (e0[k] * es) & ~(int64_t)15;
      const int64_t b1 = (e1[k] * es + 15) & ~(int64_t)15;
      const int64_t end = (T[k].nnz * es) & ~(int64_t)15;  // last whole 16-byte block of the array
      const int64_t nb = b1 - b0;
      if (b1 > end || nb < 0 || nb > (int64_t)kSlotBytes) fits = false;  // (nb < 0: rows out of order)
      L.b0[q] = b0;
      L.len[q] = (nb >= 0 && nb <= (int64_t)kSlotBytes) ? (uint32_t)nb : 0u;
      off += L.len[q];
    }
  }
  L.total = off;
  L.fits = fits && off <= (uint32_t)kSlotBytes;
}

// One lane: arrive on the slot's barrier expecting the tile's bytes and start the copies (an empty
// arrival for a tile read from global memory).
__device__ __forceinline__ void issue(const Term *T, int nt, const Lay &L, unsigned char *slot, uint64_t *bar) {
  tc::mbar_expect_tx(bar, L.fits ? L.total : 0u);
  if (!L.fits) return;
#pragma unroll
  for (int k = 0; k < kMaxTerms; k++) {
    if (k >= nt) continue;
    if (L.len[2 * k]) tc::bulk_load(slot + L.off[2 * k], (const char *)T[k].col + L.b0[2 * k], L.len[2 * k], bar);
    if (L.len[2 * k + 1])
      tc::bulk_load(slot + L.off[2 * k + 1], (const char *)T[k].fval + L.b0[2 * k + 1], L.len[2 * k + 1], bar);
  }
}

// bounded wait on an mbarrier phase (global timer), false if it runs out
__device__ __forceinline__ bool wait_slot(uint64_t *bar, uint32_t parity, long long limit_ns) {
  if (tc::mbar_try_wait(bar, parity)) return true;
  const long long t0 = globaltimer_ns();
  for (unsigned spin = 0;; spin++) {
    if (tc::mbar_try_wait(bar, parity)) return true;
    if ((spin & 63u) == 63u && (globaltimer_ns() - t0 > limit_ns || spin > (1u << 26))) return false;
  }
}

// Per-warp pipeline state (the same in every lane of the warp).  Consumption n of the warp reads
// slot n & 1 (phase parity (n >> 1) & 1) and holds the warp's tile n mod ntiles; after consuming n
// the warp issues n + 2.
struct Pipe {
  unsigned char *slot0;
  uint64_t *bar;            // two mbarriers in shared memory
  long long issued, consumed;
  int ntiles;               // tiles of this warp per pass (0: the warp has no rows)
  int w;                    // warp index in the CTA
  bool primed;
  // row data of the next tile to consume, loaded one tile ahead: per term the row's entry range
  // and (product terms) its exponent
  int64_t ne0[kMaxTerms], ne1[kMaxTerms];
  int nfe[kMaxTerms];
};

__device__ __forceinline__ void tile_rows(const Pipe &P, int64_t lo, int64_t hi, long long n, int64_t &ra,
                                          int64_t &rb) {
  const int64_t t = P.w + (int64_t)kWarps * (n % P.ntiles);
  ra = lo + kTile * t;
  rb = min(hi, ra + kTile);
}

// entry ranges and exponents of this lane's row r of tile consumption n (zero-length if r >= rb)
__device__ __forceinline__ void load_rowdata(Pipe &P, const Term *T, int nt, int64_t r, int64_t rb) {
#pragma unroll
  for (int k = 0; k < kMaxTerms; k++) {
    P.ne0[k] = P.ne1[k] = 0;
    P.nfe[k] = 0;
    if (k >= nt || r >= rb) continue;
    term_span(T[k], r, r + 1, P.ne0[k], P.ne1[k]);
    if (!T[k].pattern) P.nfe[k] = __ldg(T[k].fexp + r);
  }
}

// the runs' entry ranges of consumption n (row pointers loaded here)
__device__ __forceinline__ void tile_spans(const Pipe &P, const Term *T, int nt, int64_t lo, int64_t hi, long long n,
                                           int64_t (&e0)[kMaxTerms], int64_t (&e1)[kMaxTerms]) {
  int64_t ra, rb;
  tile_rows(P, lo, hi, n, ra, rb);
#pragma unroll
  for (int k = 0; k < kMaxTerms; k++) {
    e0[k] = e1[k] = 0;
    if (k < nt) term_span(T[k], ra, rb, e0[k], e1[k]);
  }
}

// lane 0 of the warp: copy the runs of consumption n (entry ranges e0, e1) into its slot
__device__ __forceinline__ void issue_tile(Pipe &P, const Term *T, int nt, long long n, const int64_t (&e0)[kMaxTerms],
                                           const int64_t (&e1)[kMaxTerms]) {
  Lay L;
  layout(T, nt, e0, e1, L);
  issue(T, nt, L, P.slot0 + (size_t)(n & 1) * kSlotBytes, P.bar + (n & 1));
}
__device__ __forceinline__ void issue_tile(Pipe &P, const Term *T, int nt, int64_t lo, int64_t hi, long long n) {
  int64_t e0[kMaxTerms], e1[kMaxTerms];
  tile_spans(P, T, nt, lo, hi, n, e0, e1);
  issue_tile(P, T, nt, n, e0, e1);
}

// Set up the warp's two mbarriers (once per kernel).
__device__ __forceinline__ void init(Pipe &P, unsigned char *smem, uint64_t *bars, int w, int lane, int64_t lo,
                                     int64_t hi) {
  P.w = w;
  P.slot0 = smem + (size_t)w * 2 * kSlotBytes;
  P.bar = bars + 2 * w;
  P.issued = P.consumed = 0;
  P.primed = false;
  const int64_t T = (hi - lo + kTile - 1) / kTile;
  P.ntiles = (int)(w < T ? (T - w + kWarps - 1) / kWarps : 0);
  if (lane == 0) {
    tc::mbar_init(P.bar, 1);
    tc::mbar_init(P.bar + 1, 1);
    tc::mbar_fence_init();
  }
  __syncwarp();
}

// Wait (bounded) for every copy still in flight: before the kernel returns.
__device__ __forceinline__ void drain(Pipe &P, long long limit_ns) {
  for (long long n = P.consumed; n < P.issued; n++) wait_slot(P.bar + (n & 1), (uint32_t)((n >> 1) & 1), limit_ns);
  P.consumed = P.issued;
}

// sum over the lane's row of Z[col] (pattern term), columns in shared memory at cs
__device__ __forceinline__ longlong2 zsum_smem(const int32_t *cs, int len, const longlong2 *z, bool vec4) {
  longlong2 acc = make_longlong2(0, 0);
  int k = 0;
  if (vec4) {  // 16-byte aligned rows whose length is a multiple of 4 (rows of one length)
    for (; k + kRound <= len; k += kRound) {
      int c[kRound];
#pragma unroll
      for (int q = 0; q < kRound; q += 4) {
        const int4 v = *reinterpret_cast<const int4 *>(cs + k + q);
        c[q] = v.x; c[q + 1] = v.y; c[q + 2] = v.z; c[q + 3] = v.w;
      }
      longlong2 g[kRound];
#pragma unroll
      for (int q = 0; q < kRound; q++) g[q] = rows::ldz(z + c[q]);
#pragma unroll
      for (int q = 0; q < kRound; q++) rows::zadd(acc, g[q]);
    }
    for (; k + 4 <= len; k += 4) {
      const int4 v = *reinterpret_cast<const int4 *>(cs + k);
      const longlong2 g0 = rows::ldz(z + v.x), g1 = rows::ldz(z + v.y), g2 = rows::ldz(z + v.z), g3 = rows::ldz(z + v.w);
      rows::zadd(acc, g0); rows::zadd(acc, g1); rows::zadd(acc, g2); rows::zadd(acc, g3);
    }
  }
  // warp-uniform trip count: lanes past their row's end add zeros
  const int lmax = __reduce_max_sync(__activemask(), len);
  for (; k < lmax; k += 8) {
    longlong2 g[8];
#pragma unroll
    for (int q = 0; q < 8; q++) g[q] = (k + q < len) ? rows::ldz(z + cs[k + q]) : make_longlong2(0, 0);
#pragma unroll
    for (int q = 0; q < 8; q++) rows::zadd(acc, g[q]);
  }
  return acc;
}

// sum over the lane's row of hi64(fval[e] Z[col[e]]) (product term), columns at cs and mantissas at
// vs in shared memory, with the warp's longest row as the trip count
__device__ __forceinline__ longlong2 zprod_smem(const int32_t *cs, const long long *vs, int len, const longlong2 *z) {
  const int lmax = __reduce_max_sync(__activemask(), len);
  longlong2 acc = make_longlong2(0, 0);
  for (int k = 0; k < lmax; k += kRound) {
    longlong2 g[kRound];
    long long a[kRound];
#pragma unroll
    for (int q = 0; q < kRound; q++) {
      const bool in = k + q < len;
      a[q] = in ? vs[k + q] : 0ll;
      g[q] = in ? rows::ldz(z + cs[k + q]) : make_longlong2(0, 0);
    }
#pragma unroll
    for (int q = 0; q < kRound; q++) {
      acc.x += __mul64hi(a[q], g[q].x);
      acc.y += __mul64hi(a[q], g[q].y);
    }
  }
  return acc;
}

}  // namespace stage
}  // namespace mg
