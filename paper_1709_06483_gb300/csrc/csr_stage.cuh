// Staged rows for the fixed-point Leja pass (FAM_CSR, linear generators, row_layout STAGED): each
// warp takes the block's rows in tiles of 32 (one row per lane; a tile is one slice of the sliced
// rows, slices.cu) and reads the matrix of its sliced terms from shared memory.  The slice's head
// (w entries per row, column-major) and the tile's tail entries (row-major) are contiguous runs of
// the sliced arrays, so one lane copies them into a slot of the warp's shared memory with
// cp.async.bulk (the TMA bulk engine) two tiles ahead of the tile the warp computes, completion
// counted on the slot's mbarrier, and writes a small descriptor of the slot beside it.  The lanes
// then read entry k of their 32 rows from consecutive words (no bank conflicts) and only gather the
// fixed-point vector from global memory.  Rows of one length of a pattern term (plen, the
// transverse field) need no row pointer: their columns are read from global memory with 16-byte
// loads issued at the start of the tile.  The matrix is the same in every Leja iteration, so the
// pipeline runs on across iterations: the copies issued at the end of a pass are the first tiles
// of the next one.
//
// Sums and products are exact 64-bit integers (rows.cuh), so the order in which a row's entries are
// read does not change the result: a staged row gives the bits of the sliced and CSR rows.  A tile
// whose runs do not fit a slot is read from global memory by the sliced rows (its copy is an empty
// arrival).  The sliced tail arrays carry 16 bytes of padding, so a run rounded out to whole
// 16-byte blocks stays inside them.
#pragma once

#include "rows.cuh"
#include "tcgen05.cuh"

namespace mg {
namespace stage {

constexpr int kWarps = 8;            // warps per CTA (256 threads), two CTAs per SM
constexpr int kTile = 32;            // rows per tile (one slice), one per lane
constexpr int kSlotBytes = 6400;     // 50 x 128 B: the 20-spin chain's H_s tiles need up to 6,752
constexpr int kDescBytes = 128;      // two descriptors of a warp's slots, then its next span
constexpr int kTerms = 2;            // terms of a staged plan (the register arrays are this long)
constexpr size_t kSmemBytes = (size_t)kWarps * (2 * kSlotBytes + 3 * kDescBytes);  // 105,472 B per CTA

__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// a term read from the slots: sliced, and not a pattern whose rows are all one length
__device__ __forceinline__ bool staged_term(const Term &t) { return t.hbase && !(t.pattern && t.plen); }

// Slot descriptor (written by lane 0 at issue time, read by the lanes after the slot's phase).
struct Desc {
  int fits;
  int w[kTerms];             // head width of each staged term in this slice
  uint32_t hc[kTerms];       // slot offsets: head columns, head mantissas,
  uint32_t hv[kTerms];
  uint32_t tc[kTerms];       // the tail runs (their first 16-byte block)
  uint32_t tv[kTerms];
  long long t0[kTerms];      // first tail entry of the tile
};
static_assert(sizeof(Desc) <= kDescBytes, "descriptor size");

// Runs of one tile: slice s = ra / 32; per staged term the head [hbase[s], hbase[s+1]) and the tail
// entries [tptr[ra], tptr[rb]).
struct Span {
  long long h0[kTerms], h1[kTerms], t0[kTerms], t1[kTerms];
};
static_assert(sizeof(Span) <= kDescBytes, "span size");

__device__ __forceinline__ void load_span(const Term *T, int nt, int64_t ra, int64_t rb, Span &S) {
#pragma unroll
  for (int k = 0; k < kTerms; k++) {
    S.h0[k] = S.h1[k] = S.t0[k] = S.t1[k] = 0;
    if (k >= nt || !staged_term(T[k])) continue;
    S.h0[k] = __ldg(T[k].hbase + (ra >> 5));
    S.h1[k] = __ldg(T[k].hbase + (ra >> 5) + 1);
    if (T[k].tptr) {
      S.t0[k] = __ldg(T[k].tptr + ra);
      S.t1[k] = __ldg(T[k].tptr + rb);
    }
  }
}

// tail run of entries [t0, t1) of `es`-byte entries, rounded out to whole 16-byte blocks
__device__ __forceinline__ long long run_lo(long long t0, int es) { return (t0 * es) & ~15ll; }
__device__ __forceinline__ long long run_hi(long long t1, int es) { return (t1 * es + 15) & ~15ll; }

// Slot layout of a tile; returns its bytes (D.fits: they fit one slot).
__device__ __forceinline__ uint32_t layout(const Term *T, int nt, const Span &S, Desc &D) {
  long long off = 0;
  bool ok = true;
#pragma unroll
  for (int k = 0; k < kTerms; k++) {
    D.w[k] = 0;
    D.hc[k] = D.hv[k] = D.tc[k] = D.tv[k] = 0;
    D.t0[k] = 0;
    if (k >= nt || !staged_term(T[k])) continue;
    const long long nh = S.h1[k] - S.h0[k];  // 32 w entries
    const long long nl = S.t1[k] - S.t0[k];
    if (nh < 0 || nh > kSlotBytes || nl < 0 || nl > kSlotBytes) { ok = false; continue; }  // (malformed)
    D.w[k] = (int)(nh >> 5);
    D.t0[k] = S.t0[k];
    D.hc[k] = (uint32_t)off;
    off += 4 * nh;
    if (!T[k].pattern) {
      D.hv[k] = (uint32_t)off;
      off += 8 * nh;
    }
    if (T[k].tptr && nl > 0) {
      D.tc[k] = (uint32_t)off;
      off += run_hi(S.t1[k], 4) - run_lo(S.t0[k], 4);
      if (!T[k].pattern) {
        D.tv[k] = (uint32_t)off;
        off += run_hi(S.t1[k], 8) - run_lo(S.t0[k], 8);
      }
    }
  }
  D.fits = ok && off <= kSlotBytes;
  return (uint32_t)(D.fits ? off : 0);
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
  unsigned char *slot0;     // two slots, then two descriptors
  uint64_t *bar;            // two mbarriers in shared memory
  long long issued, consumed;
  int ntiles;               // tiles of this warp per pass (0: the warp has no rows)
  int w;                    // warp index in the CTA
  int tc;                   // consumed mod ntiles (the tile of the next consumption)
  bool primed;
  // row data of the next tile to consume, loaded one tile ahead: per staged term the row's tail
  // range, per product term its exponent
  long long nt0[kTerms], nt1[kTerms];
  int nfe[kTerms];
};

__device__ __forceinline__ unsigned char *slot_ptr(const Pipe &P, long long n) {
  return P.slot0 + (size_t)(n & 1) * kSlotBytes;
}
__device__ __forceinline__ Desc *desc_ptr(const Pipe &P, long long n) {
  return reinterpret_cast<Desc *>(P.slot0 + 2 * (size_t)kSlotBytes + (size_t)(n & 1) * kDescBytes);
}
// lane 0's record of the runs of the tile it copies next (shared memory, not registers)
__device__ __forceinline__ Span *span_ptr(const Pipe &P) {
  return reinterpret_cast<Span *>(P.slot0 + 2 * (size_t)kSlotBytes + 2 * (size_t)kDescBytes);
}

// rows of the warp's tile `i` (0 <= i < ntiles)
__device__ __forceinline__ void tile_rows(const Pipe &P, int64_t lo, int64_t hi, int i, int64_t &ra, int64_t &rb) {
  ra = lo + (int64_t)kTile * (P.w + kWarps * i);
  rb = min(hi, ra + kTile);
}
// tile index d consumptions after the next one (d small): no division
__device__ __forceinline__ int tile_ahead(const Pipe &P, int d) {
  int i = P.tc + d;
  while (i >= P.ntiles) i -= P.ntiles;
  return i;
}

// tail range and exponent of this lane's row r (zero-length if r >= rb)
__device__ __forceinline__ void load_rowdata(Pipe &P, const Term *T, int nt, int64_t r, int64_t rb) {
#pragma unroll
  for (int k = 0; k < kTerms; k++) {
    P.nt0[k] = P.nt1[k] = 0;
    P.nfe[k] = 0;
    if (k >= nt || r >= rb) continue;
    if (!T[k].pattern) P.nfe[k] = __ldg(T[k].fexp + r);
    if (staged_term(T[k]) && T[k].tptr) {
      P.nt0[k] = __ldg(T[k].tptr + r);
      P.nt1[k] = __ldg(T[k].tptr + r + 1);
    }
  }
}

// lane 0: write the descriptor of consumption n and start its copies (an empty arrival if the tile
// does not fit)
__device__ __forceinline__ void issue(Pipe &P, const Term *T, int nt, long long n, const Span &S) {
  Desc L;
  const uint32_t total = layout(T, nt, S, L);
  *desc_ptr(P, n) = L;
  unsigned char *slot = slot_ptr(P, n);
  uint64_t *bar = P.bar + (n & 1);
  tc::mbar_expect_tx(bar, total);
  if (!L.fits) return;
#pragma unroll
  for (int k = 0; k < kTerms; k++) {
    if (k >= nt || !staged_term(T[k])) continue;
    const uint32_t nh = (uint32_t)(S.h1[k] - S.h0[k]);
    if (nh) {
      tc::bulk_load(slot + L.hc[k], T[k].hcol + S.h0[k], 4 * nh, bar);
      if (!T[k].pattern) tc::bulk_load(slot + L.hv[k], T[k].hval + S.h0[k], 8 * nh, bar);
    }
    if (T[k].tptr && S.t1[k] > S.t0[k]) {
      const long long b0 = run_lo(S.t0[k], 4), b1 = run_hi(S.t1[k], 4);
      tc::bulk_load(slot + L.tc[k], (const char *)T[k].tcol + b0, (uint32_t)(b1 - b0), bar);
      if (!T[k].pattern) {
        const long long v0 = run_lo(S.t0[k], 8), v1 = run_hi(S.t1[k], 8);
        tc::bulk_load(slot + L.tv[k], (const char *)T[k].tval + v0, (uint32_t)(v1 - v0), bar);
      }
    }
  }
}

// Set up the warp's two mbarriers (once per kernel).
__device__ __forceinline__ void init(Pipe &P, unsigned char *smem, uint64_t *bars, int w, int lane, int64_t lo,
                                     int64_t hi) {
  P.w = w;
  P.slot0 = smem + (size_t)w * (2 * kSlotBytes + 3 * kDescBytes);
  P.bar = bars + 2 * w;
  P.issued = P.consumed = 0;
  P.tc = 0;
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

// sum over the lane's staged row of Z[col] (pattern term): head entry k at hc[32 k], tail at tc
__device__ __forceinline__ longlong2 zsum_staged(const int32_t *hc, int w, const int32_t *tc, int tlen,
                                                 const longlong2 *z) {
  longlong2 acc = make_longlong2(0, 0);
  int k = 0;
  for (; k + 8 <= w; k += 8) {
    longlong2 g[8];
#pragma unroll
    for (int q = 0; q < 8; q++) g[q] = rows::ldz(z + hc[32 * (k + q)]);
#pragma unroll
    for (int q = 0; q < 8; q++) rows::zadd(acc, g[q]);
  }
  for (; k < w; k++) rows::zadd(acc, rows::ldz(z + hc[32 * k]));
  for (int j = 0; j < tlen; j++) rows::zadd(acc, rows::ldz(z + tc[j]));
  return acc;
}

// sum over the lane's staged row of hi64(a Z[col]) (product term): head mantissa k at hv[32 k], the
// tail's at tv; the tail with the warp's longest tail as the trip count (call with the warp converged)
__device__ __forceinline__ longlong2 zprod_staged(const int32_t *hc, const long long *hv, int w, const int32_t *tc,
                                                  const long long *tv, int tlen, const longlong2 *z) {
  longlong2 acc = make_longlong2(0, 0);
  int k = 0;
  for (; k + 8 <= w; k += 8) {
    long long a[8];
    longlong2 g[8];
#pragma unroll
    for (int q = 0; q < 8; q++) {
      a[q] = hv[32 * (k + q)];
      g[q] = rows::ldz(z + hc[32 * (k + q)]);
    }
#pragma unroll
    for (int q = 0; q < 8; q++) {
      acc.x += __mul64hi(a[q], g[q].x);
      acc.y += __mul64hi(a[q], g[q].y);
    }
  }
  for (; k < w; k++) {
    const long long a = hv[32 * k];
    const longlong2 g = rows::ldz(z + hc[32 * k]);
    acc.x += __mul64hi(a, g.x);
    acc.y += __mul64hi(a, g.y);
  }
  const int lmax = __reduce_max_sync(__activemask(), tlen);
  for (int j = 0; j < lmax; j += 4) {
    long long a[4];
    longlong2 g[4];
#pragma unroll
    for (int q = 0; q < 4; q++) {
      const bool in = j + q < tlen;
      a[q] = in ? tv[j + q] : 0ll;
      g[q] = in ? rows::ldz(z + tc[j + q]) : make_longlong2(0, 0);
    }
#pragma unroll
    for (int q = 0; q < 4; q++) {
      acc.x += __mul64hi(a[q], g[q].x);
      acc.y += __mul64hi(a[q], g[q].y);
    }
  }
  return acc;
}

}  // namespace stage
}  // namespace mg
