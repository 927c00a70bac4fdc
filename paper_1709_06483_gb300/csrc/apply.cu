// y = sum_k beta_k H_k x for every state of a plan: the generator matvec of the Leja recurrence
// (arXiv:1709.06483, Sec. 3, where these products make up the cost of the method) as a call of its own,
// for expectation values and for timing the matvec outside the propagation.  CSR, matrix-free and
// mixed terms use the same row code as the persistent kernel (rows.cuh); dense terms one warp per
// row and state.
//
// Plans with fixed-point arithmetic take the matvec as the Leja iteration does: max |x| per state
// (k_apply_absmax), the copy Z = trunc(x 2^s) with s from that bound (k_apply_fix), then the rows
// with the pattern sums and value products on Z (k_apply<FAM, true>); three launches, the FP64
// pipe left with the per-row conversions.
#include <cuda_runtime.h>

#include "magnus_internal.cuh"
#include "persist_common.cuh"
#include "rows.cuh"

namespace mg {
namespace {

using namespace rows;

struct Beta {
  double b[kMaxTerms];
};

// fixed-point rows: registers capped as in the persistent kernel's fixed-point instantiation (4
// resident CTAs per SM for CSR, 3 for the matrix-free chain); 0 = no occupancy hint (FP64 rows)
template <int FAM, bool ZF>
constexpr int apply_min_blocks() {
  return ZF ? (FAM == FAM_CSR ? 4 : 3) : 0;
}

// the two passes over x take kPassRows rows per thread (loads issued together, coalesced), grid
// (ceil(D / (256 kPassRows)), nv)
constexpr int kPassRows = 4;

// m[v] = max over the rows of state v of abshi(x) (m zeroed by the launcher); one atomic per
// block (atomics of every warp on the one word serialise at L2)
__global__ void __launch_bounds__(256) k_apply_absmax(const double2 *x, int64_t D, unsigned *m) {
  __shared__ unsigned s_h[8];
  const double2 *xv = x + (int64_t)blockIdx.y * D;
  const int64_t r0 = (int64_t)blockIdx.x * blockDim.x * kPassRows + threadIdx.x;
  unsigned h = 0;
#pragma unroll
  for (int u = 0; u < kPassRows; u++) {
    const int64_t r = r0 + (int64_t)u * blockDim.x;
    if (r < D) h = max(h, abshi(xv[r]));
  }
  h = __reduce_max_sync(0xFFFFFFFFu, h);
  if ((threadIdx.x & 31) == 0) s_h[threadIdx.x >> 5] = h;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < 8; w++) h = max(h, s_h[w]);
    if (h) atomicMax(m + blockIdx.y, h);
  }
}

// Z copy of state v at the scale of its bound (a state with a non-finite entry is left to the
// FP64 rows)
__global__ void __launch_bounds__(256) k_apply_fix(const double2 *x, int64_t D, const unsigned *m, int hb,
                                                   longlong2 *z) {
  const unsigned h = m[blockIdx.y];
  if (h >= 0x7FF00000u) return;
  const int zs = fix_scale(abshi_bound(h), hb);
  const int64_t off = (int64_t)blockIdx.y * D;
  const int64_t r0 = (int64_t)blockIdx.x * blockDim.x * kPassRows + threadIdx.x;
#pragma unroll
  for (int u = 0; u < kPassRows; u++) {
    const int64_t r = r0 + (int64_t)u * blockDim.x;
    if (r < D) z[off + r] = fix2(x[off + r], zs);
  }
}

template <int FAM, bool ZF>
__global__ void __launch_bounds__(256, apply_min_blocks<FAM, ZF>())
    k_apply(const Term *terms, int nt, Beta beta, int lbits, const double *dlo, const double *dhi, const double2 *x,
            double2 *y, int64_t D, int nv, const longlong2 *z, const unsigned *zmax, int hb) {
  __shared__ Term sT[kMaxTerms];
  __shared__ ExpRec sR;
  __shared__ double s_jb[kMaxSpins], s_j2[kMaxSpins];
  __shared__ double s_wz[kMaxTerms];     // fixed point: weights of the pattern sums, beta_k v_k
  __shared__ long long s_cb[kMaxSpins];  // fixed point, matrix-free: bond weights as 62-bit mantissas
  __shared__ int s_cbe;
  const int tid = threadIdx.x;
  for (int i = tid; i < nt * (int)sizeof(Term) / 4; i += blockDim.x)
    reinterpret_cast<int *>(sT)[i] = reinterpret_cast<const int *>(terms)[i];
  if (tid == 0)
    for (int k = 0; k < kMaxTerms; k++) sR.bg[k] = (k < nt) ? beta.b[k] : 0.0;
  __syncthreads();
  if (ZF && tid < nt) s_wz[tid] = beta.b[tid] * sT[tid].pval;
  Ctx cx{};
  cx.T = sT;
  cx.nt = nt;
  cx.n = sT[0].nspins;
  cx.lbits = lbits;
  cx.lomask = ((int64_t)1 << (lbits + 1)) - 1;
  cx.dlo = dlo;
  cx.dhi = dhi;
  cx.jb = s_jb;
  cx.j2 = s_j2;
  if (FAM == FAM_MF) {
    for (int p = 1 + tid; p < cx.n; p += blockDim.x) {
      s_j2[p - 1] = 2.0 * sT[0].J[cx.n - p - 1];
      s_jb[p - 1] = s_j2[p - 1] * beta.b[0];
    }
    __syncthreads();
    if (ZF) {  // bond weights 2 J beta_0 as mantissas at one exponent E: max |w| < 2^E
      if (tid == 0) {
        double wmax = 0.0;
        for (int p = 0; p < cx.n - 1; p++) wmax = fmax(wmax, fabs(s_jb[p]));
        int E = 0;
        if (wmax > 0.0) frexp(wmax, &E);
        E = max(-400, min(400, E));
        for (int p = 0; p < cx.n - 1; p++) s_cb[p] = llrint(ldexp(s_jb[p], 62 - E));
        s_cbe = E;
      }
      __syncthreads();
      cx.cb = s_cb;
      cx.cbe = s_cbe;
    }
  }
  __syncthreads();
  const int64_t total = (int64_t)nv * D;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + tid; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = i / D, r = i - v * D;
    double2 xr;
    if constexpr (ZF) {
      const unsigned h = zmax[v];
      if (h < 0x7FF00000u) {
        y[i] = Op<FAM>::combo_z(cx, sR, s_wz, 0.0, x + v * D, z + v * D, fix_scale(abshi_bound(h), hb), r, xr);
        continue;
      }
    }
    y[i] = Op<FAM>::combo(cx, sR, 0.0, x + v * D, r, xr);
  }
}

// dense terms (and transverse-field terms mixed with them): one warp per (state, row)
__global__ void __launch_bounds__(256) k_apply_dense(const Term *terms, int nt, Beta beta, const double2 *x,
                                                     double2 *y, int64_t D, int nv) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t w = w0; w < (int64_t)nv * D; w += nw) {
    const int64_t v = w / D, r = w - v * D;
    const double2 *xv = x + v * D;
    double2 acc = make_double2(0.0, 0.0);
    for (int k = 0; k < nt; k++) {
      const Term &t = terms[k];
      double2 part = make_double2(0.0, 0.0);
      if (t.kind == MAGNUS_TERM_DENSE) {
        if (t.real_valued)
          for (int64_t j = lane; j < D; j += 32) part = rfma(t.rv[(r * D + j) * t.rs], xv[j], part);
        else
          for (int64_t j = lane; j < D; j += 32) part = cfma(t.val[r * D + j], xv[j], part);
      } else if (lane == 0) {
        part = term_row_generic(t, xv, r);
      }
      acc = rfma(beta.b[k], part, acc);
    }
    acc.x = warp_sum(acc.x);
    acc.y = warp_sum(acc.y);
    if (lane == 0) y[w] = acc;
  }
}

}  // namespace

cudaError_t launch_apply(int fam, const Term *terms, int nt, const double *beta, int lbits, const double *dlo,
                         const double *dhi, const double2 *x, double2 *y, int64_t D, int nv, longlong2 *zc,
                         unsigned *zmax, int zhb, int num_sms, cudaStream_t st) {
  Beta b{};
  for (int k = 0; k < nt && k < kMaxTerms; k++) b.b[k] = beta[k];
  const int grid = num_sms * 8;
  if (zc && zmax && (fam == FAM_CSR || fam == FAM_MF)) {
    cudaError_t e = cudaMemsetAsync(zmax, 0, sizeof(unsigned) * nv, st);
    if (e != cudaSuccess) return e;
    const dim3 g2((unsigned)((D + 256 * kPassRows - 1) / (256 * kPassRows)), (unsigned)nv);
    k_apply_absmax<<<g2, 256, 0, st>>>(x, D, zmax);
    k_apply_fix<<<g2, 256, 0, st>>>(x, D, zmax, zhb, zc);
    // the rows: one wave of resident blocks
    if (fam == FAM_CSR)
      k_apply<FAM_CSR, true><<<num_sms * apply_min_blocks<FAM_CSR, true>(), 256, 0, st>>>(
          terms, nt, b, lbits, dlo, dhi, x, y, D, nv, zc, zmax, zhb);
    else
      k_apply<FAM_MF, true><<<num_sms * apply_min_blocks<FAM_MF, true>(), 256, 0, st>>>(
          terms, nt, b, lbits, dlo, dhi, x, y, D, nv, zc, zmax, zhb);
    return cudaGetLastError();
  }
  switch (fam) {
    case FAM_CSR:
      k_apply<FAM_CSR, false><<<grid, 256, 0, st>>>(terms, nt, b, lbits, dlo, dhi, x, y, D, nv, nullptr, nullptr, 0);
      break;
    case FAM_MF:
      k_apply<FAM_MF, false><<<grid, 256, 0, st>>>(terms, nt, b, lbits, dlo, dhi, x, y, D, nv, nullptr, nullptr, 0);
      break;
    case FAM_DENSE: k_apply_dense<<<grid, 256, 0, st>>>(terms, nt, b, x, y, D, nv); break;
    default:
      k_apply<FAM_GENERIC, false><<<grid, 256, 0, st>>>(terms, nt, b, lbits, dlo, dhi, x, y, D, nv, nullptr, nullptr,
                                                         0);
      break;
  }
  return cudaGetLastError();
}

}  // namespace mg
