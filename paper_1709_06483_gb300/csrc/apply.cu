// y = sum_k beta_k H_k x for every state of a plan: the generator matvec of the Leja recurrence
// (arXiv:1709.06483, Sec. 3, where these products make up the cost of the method) as a call of its own,
// for expectation values and for timing the matvec outside the propagation.  CSR, matrix-free and
// mixed terms use the same row code as the persistent kernel (rows.cuh); dense terms one warp per
// row and state.
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

template <int FAM>
__global__ void __launch_bounds__(256) k_apply(const Term *terms, int nt, Beta beta, int lbits, const double *dlo,
                                               const double *dhi, const double2 *x, double2 *y, int64_t D, int nv) {
  __shared__ Term sT[kMaxTerms];
  __shared__ ExpRec sR;
  __shared__ double s_jb[kMaxSpins], s_j2[kMaxSpins];
  const int tid = threadIdx.x;
  for (int i = tid; i < nt * (int)sizeof(Term) / 4; i += blockDim.x)
    reinterpret_cast<int *>(sT)[i] = reinterpret_cast<const int *>(terms)[i];
  if (tid == 0)
    for (int k = 0; k < kMaxTerms; k++) sR.bg[k] = (k < nt) ? beta.b[k] : 0.0;
  __syncthreads();
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
  }
  const int64_t total = (int64_t)nv * D;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + tid; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = i / D, r = i - v * D;
    double2 xr;
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
                         const double *dhi, const double2 *x, double2 *y, int64_t D, int nv, int num_sms,
                         cudaStream_t st) {
  Beta b{};
  for (int k = 0; k < nt && k < kMaxTerms; k++) b.b[k] = beta[k];
  const int grid = num_sms * 8;
  switch (fam) {
    case FAM_CSR: k_apply<FAM_CSR><<<grid, 256, 0, st>>>(terms, nt, b, lbits, dlo, dhi, x, y, D, nv); break;
    case FAM_MF: k_apply<FAM_MF><<<grid, 256, 0, st>>>(terms, nt, b, lbits, dlo, dhi, x, y, D, nv); break;
    case FAM_DENSE: k_apply_dense<<<grid, 256, 0, st>>>(terms, nt, b, x, y, D, nv); break;
    default: k_apply<FAM_GENERIC><<<grid, 256, 0, st>>>(terms, nt, b, lbits, dlo, dhi, x, y, D, nv); break;
  }
  return cudaGetLastError();
}

}  // namespace mg
