// Sliced rows of a CSR term, built once at plan creation for the fixed-point rows (rows.cuh).
//
// A slice is 32 consecutive rows, one per lane of the warp that computes them.  Its head holds the
// first w entries of every row, w the slice's shortest row, column-major: entry k of lane l at
// 32 k + l, so that the warp loads entry k of its 32 rows in one coalesced access and needs no row
// pointer for them.  The rest of each row (its tail: most rows of a banded or spin-chain matrix
// have none or a few entries there) stays row-major behind a row pointer.  The entries of a row
// are ordered by how many rows of the slice hold the same column offset col - r (most first, then
// by offset), so that where the matrix has the same structure from row to row -- a spin chain's
// flips of the high bits, the bands of a banded matrix -- entry k of the 32 rows reads one run of
// the vector.  The fixed-point row sums are exact integers, so the order of a row's entries does not
// change any result.  Same bytes as the CSR arrays, plus 8 B per 32 rows.
#include <cuda_runtime.h>

#include <algorithm>

#include "magnus_internal.cuh"

namespace mg {
namespace {

constexpr int kSortCap = 24;       // rows of a slice all at most this long are ordered
constexpr int kFillWarps = 4;      // warps (slices) per block of the fill kernel

// w[s] = shortest row of slice s (its rows < dim)
__global__ void k_slice_width(const int64_t *rowptr, int64_t dim, int64_t nslice, int64_t *w) {
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < nslice; s += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r0 = s * 32, r1 = min(dim, r0 + 32);
    int64_t m = INT64_MAX;
    for (int64_t r = r0; r < r1; r++) m = min(m, rowptr[r + 1] - rowptr[r]);
    w[s] = 32 * m;  // head entries of the slice
  }
}

// t[r] = entries of row r beyond its slice's head width
__global__ void k_tail_len(const int64_t *rowptr, int64_t dim, const int64_t *w, int64_t *t) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < dim; r += (int64_t)gridDim.x * blockDim.x)
    t[r] = (rowptr[r + 1] - rowptr[r]) - w[r >> 5] / 32;
}

// out[0] = 0, out[i+1] = in[0] + ... + in[i] (one block: each thread sums a contiguous chunk, the
// chunk sums are scanned in shared memory, then every thread writes its chunk's prefixes)
__global__ void k_scan(const int64_t *in, int64_t n, int64_t *out) {
  __shared__ int64_t part[1024];
  const int t = threadIdx.x, T = blockDim.x;
  const int64_t chunk = (n + T - 1) / T;
  const int64_t a = min(n, t * chunk), b = min(n, a + chunk);
  int64_t sum = 0;
  for (int64_t i = a; i < b; i++) sum += in[i];
  part[t] = sum;
  __syncthreads();
  if (t == 0) {
    int64_t run = 0;
    for (int i = 0; i < T; i++) {
      const int64_t v = part[i];
      part[i] = run;
      run += v;
    }
    out[n] = run;
  }
  __syncthreads();
  int64_t run = part[t];
  for (int64_t i = a; i < b; i++) {
    out[i] = run;
    run += in[i];
  }
}

// One warp per slice: order each row's entries (rows of at most kSortCap entries) and write the head
// and the tail.
__global__ void k_slice_fill(const int64_t *rowptr, const int32_t *col, const long long *fval, int64_t dim,
                             int64_t nslice, const int64_t *hbase, const int64_t *tptr, int32_t *hcol, long long *hval,
                             int32_t *tcol, long long *tval) {
  __shared__ int32_t s_col[kFillWarps][32][kSortCap];
  __shared__ long long s_val[kFillWarps][32][kSortCap];
  const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
  const int64_t s = (int64_t)blockIdx.x * kFillWarps + wl;
  if (s >= nslice) return;
  const int64_t r = s * 32 + lane;
  const bool valid = r < dim;
  const int64_t e0 = valid ? rowptr[r] : 0;
  const int len = valid ? (int)(rowptr[r + 1] - e0) : 0;
  const int64_t hb = hbase[s];
  const int w = (int)((hbase[s + 1] - hb) / 32);
  const int64_t t0 = (tptr && valid) ? tptr[r] : 0;
  const bool sortable = __all_sync(0xffffffffu, len <= kSortCap);
  int32_t *mc = s_col[wl][lane];
  long long *mv = s_val[wl][lane];
  if (sortable) {
    for (int k = 0; k < len; k++) {
      mc[k] = col[e0 + k];
      mv[k] = fval ? fval[e0 + k] : 0ll;
    }
    __syncwarp();
    // how many rows of the slice hold each of this row's column offsets
    int cnt[kSortCap];
    for (int k = 0; k < len; k++) {
      const int64_t d = (int64_t)mc[k] - r;
      int c = 0;
      for (int l2 = 0; l2 < 32; l2++) {
        const int64_t r2 = s * 32 + l2;
        if (r2 >= dim) break;
        const int n2 = (int)(rowptr[r2 + 1] - rowptr[r2]);
        for (int k2 = 0; k2 < n2; k2++)
          if ((int64_t)s_col[wl][l2][k2] - r2 == d) {
            c++;
            break;
          }
      }
      cnt[k] = c;
    }
    __syncwarp();
    // insertion sort of the lane's entries: most shared offset first, then by offset
    for (int k = 1; k < len; k++) {
      const int32_t ck = mc[k];
      const long long vk = mv[k];
      const int nk = cnt[k];
      const int64_t dk = (int64_t)ck - r;
      int j = k - 1;
      while (j >= 0 && (cnt[j] < nk || (cnt[j] == nk && (int64_t)mc[j] - r > dk))) {
        mc[j + 1] = mc[j];
        mv[j + 1] = mv[j];
        cnt[j + 1] = cnt[j];
        j--;
      }
      mc[j + 1] = ck;
      mv[j + 1] = vk;
      cnt[j + 1] = nk;
    }
    for (int k = 0; k < len; k++) {
      if (k < w) {
        hcol[hb + 32 * k + lane] = mc[k];
        if (hval) hval[hb + 32 * k + lane] = mv[k];
      } else {
        tcol[t0 + k - w] = mc[k];
        if (tval) tval[t0 + k - w] = mv[k];
      }
    }
  } else {  // long rows: CSR order
    for (int k = 0; k < len; k++) {
      if (k < w) {
        hcol[hb + 32 * k + lane] = col[e0 + k];
        if (hval) hval[hb + 32 * k + lane] = fval[e0 + k];
      } else {
        tcol[t0 + k - w] = col[e0 + k];
        if (tval) tval[t0 + k - w] = fval[e0 + k];
      }
    }
  }
  if (!valid)  // lanes past the last row: a defined head (never read by a row computation)
    for (int k = 0; k < w; k++) {
      hcol[hb + 32 * k + lane] = 0;
      if (hval) hval[hb + 32 * k + lane] = 0;
    }
}

}  // namespace

void free_sliced_rows(SlicedRows *s) {
  void *b[] = {s->hbase, s->hcol, s->hval, s->tptr, s->tcol, s->tval};
  for (void *p : b)
    if (p) cudaFree(p);
  *s = SlicedRows{};
}

cudaError_t build_sliced_rows(const int64_t *rowptr, const int32_t *col, const long long *fval, int64_t dim,
                              SlicedRows *out, cudaStream_t st) {
  *out = SlicedRows{};
  const int64_t nslice = (dim + 31) / 32;
  int64_t *w = nullptr, *tl = nullptr;
  cudaError_t e = cudaSuccess;
  auto fail = [&](cudaError_t err) {
    if (w) cudaFree(w);
    if (tl) cudaFree(tl);
    free_sliced_rows(out);
    return err;
  };
  if ((e = cudaMalloc(&w, sizeof(int64_t) * nslice)) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&out->hbase, sizeof(int64_t) * (nslice + 1))) != cudaSuccess) return fail(e);
  const int g1 = (int)std::max<int64_t>(1, std::min<int64_t>(4096, (nslice + 255) / 256));
  k_slice_width<<<g1, 256, 0, st>>>(rowptr, dim, nslice, w);
  k_scan<<<1, 1024, 0, st>>>(w, nslice, out->hbase);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail(e);
  int64_t nhead = 0, nnz = 0, first = 0;
  if ((e = cudaMemcpyAsync(&nhead, out->hbase + nslice, sizeof nhead, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(&nnz, rowptr + dim, sizeof nnz, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(&first, rowptr, sizeof first, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
      (e = cudaStreamSynchronize(st)) != cudaSuccess)
    return fail(e);
  nnz -= first;
  out->nhead = nhead;
  out->ntail = nnz - nhead;
  if ((e = cudaMalloc(&out->hcol, sizeof(int32_t) * std::max<int64_t>(1, nhead))) != cudaSuccess) return fail(e);
  if (fval && (e = cudaMalloc(&out->hval, sizeof(long long) * std::max<int64_t>(1, nhead))) != cudaSuccess)
    return fail(e);
  if (out->ntail > 0) {
    if ((e = cudaMalloc(&tl, sizeof(int64_t) * dim)) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&out->tptr, sizeof(int64_t) * (dim + 1))) != cudaSuccess) return fail(e);
    // 4 entries of padding: a run rounded out to whole 16-byte blocks (the staged rows' copies)
    // stays inside the allocation
    if ((e = cudaMalloc(&out->tcol, sizeof(int32_t) * (out->ntail + 4))) != cudaSuccess) return fail(e);
    if (fval && (e = cudaMalloc(&out->tval, sizeof(long long) * (out->ntail + 4))) != cudaSuccess) return fail(e);
    const int g2 = (int)std::max<int64_t>(1, std::min<int64_t>(4096, (dim + 255) / 256));
    k_tail_len<<<g2, 256, 0, st>>>(rowptr, dim, w, tl);
    k_scan<<<1, 1024, 0, st>>>(tl, dim, out->tptr);
  }
  const int g3 = (int)((nslice + kFillWarps - 1) / kFillWarps);
  k_slice_fill<<<g3, 32 * kFillWarps, 0, st>>>(rowptr, col, fval, dim, nslice, out->hbase, out->tptr, out->hcol,
                                               out->hval, out->tcol, out->tval);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail(e);
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return fail(e);
  cudaFree(w);
  if (tl) cudaFree(tl);
  return cudaSuccess;
}

}  // namespace mg
