// magnus_expv_xxz_static: the action exp(-i (beta_0 H_xxz + beta_1 sum_i sx_i)) v for a matrix-free
// open XXZ chain, computed without allocating any memory.  It is meant for callers that cannot call
// cudaMalloc: code whose device memory is entirely owned by another allocator or pool, and
// latency-sensitive loops that must not pay the implicit device synchronisation a cudaMalloc or
// cudaFree can cause.  All scratch lives in one fixed-size file-scope device array (g_static_scratch
// below), which every GPU that loads this library holds until the process exits.
//
// Host code must not use the name g_static_scratch as a device address (on the host it is only a
// stand-in): the device address is fetched once per device with cudaGetSymbolAddress and passed to
// the kernels.  The arithmetic is FP64 throughout: the terms go to the persistent kernel's generic
// instantiation (k_magnus_persistent<FAM_GENERIC, no M6, FP64 sums>, at least 32 rows per CTA), not to the
// matrix-free specialisation with diagonal tables and fixed-point sums that a plan chooses, so the
// two entry points round differently and agree to the Leja tolerance (tested at 1e-10), not bit for
// bit.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "magnus_internal.cuh"

namespace mg {
void noalloc_set_error(const char *msg);
}

namespace {

using namespace mg;

constexpr int kStaticMaxSpins = 16;                          // largest chain: dim 2^16 = 65,536
constexpr int64_t kStaticMaxDim = (int64_t)1 << kStaticMaxSpins;
constexpr int kStaticMmax = 100;                             // Leja degree cap, as the plan default
constexpr int kStaticMaxGrid = 2048;                         // CTAs of the persistent launch
constexpr int kStaticGershBlocks = 256;

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Byte layout of the scratch array.
constexpr size_t kOffVec = 0;                                                   // alt, w0, w1
constexpr size_t kVecBytes = align256(sizeof(double2) * kStaticMaxDim);
constexpr size_t kOffPartials = kOffVec + 3 * kVecBytes;                        // [2][grid][4]
constexpr size_t kOffTerms = kOffPartials + align256(sizeof(double) * 8 * kStaticMaxGrid);
constexpr size_t kOffTermAB = kOffTerms + align256(sizeof(Term) * 2);
constexpr size_t kOffXi = kOffTermAB + align256(sizeof(double) * 4);
constexpr size_t kOffCand = kOffXi + align256(sizeof(double) * (kStaticMmax + 1));
constexpr size_t kOffCounter = kOffCand + align256(sizeof(double) * 2 * (kStaticMmax + 1));
constexpr size_t kOffRec = kOffCounter + 256;
constexpr size_t kOffDD = kOffRec + align256(sizeof(ExpRec));
constexpr size_t kOffBar = kOffDD + align256(sizeof(double2) * (kStaticMmax + 1));
constexpr size_t kOffCounters = kOffBar + align256(sizeof(GridBar));
constexpr size_t kOffGersh = kOffCounters + align256(sizeof(Counters));
constexpr size_t kScratchBytes = kOffGersh + align256(sizeof(double) * 2 * kStaticGershBlocks);  // ~3.2 MB

static __device__ __align__(256) unsigned char g_static_scratch[kScratchBytes];

struct DeviceSetup {
  bool done = false;
  unsigned char *base = nullptr;  // device address of g_static_scratch on this device
  int num_sms = 0;
  int blocks_per_sm = 0;          // co-resident CTAs per SM of the instantiation launched below
};
std::mutex g_setup_mutex;
DeviceSetup g_setup[64];

// Writes the two matrix-free terms and clears what the kernels expect to start at zero.
__global__ void k_static_init(Term xxz, Term field, Term *terms, GridBar *bar, Counters *counters) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    terms[0] = xxz;
    terms[1] = field;
    memset(bar, 0, sizeof(GridBar));
    memset(counters, 0, sizeof(Counters));
  }
}

magnus_status fail(magnus_status s, const char *msg) {
  noalloc_set_error(msg);
  return s;
}

}  // namespace

extern "C" MAGNUS_API magnus_status magnus_expv_xxz_static(int32_t nspins, const double *J, const double *hz,
                                                            double delta, const double *beta, const void *v,
                                                            void *out, double tol, void *stream_) {
  cudaStream_t stream = (cudaStream_t)stream_;
  if (nspins < 2 || nspins > kStaticMaxSpins)
    return fail(MAGNUS_EINVAL, "magnus_expv_xxz_static: nspins must be 2..16 (the fixed scratch holds dim <= 65536)");
  if (!J || !hz || !beta || !v || !out) return fail(MAGNUS_EINVAL, "magnus_expv_xxz_static: null argument");
  if (((uintptr_t)v) % 16 || ((uintptr_t)out) % 16)
    return fail(MAGNUS_EINVAL, "magnus_expv_xxz_static: vectors must be 16-byte aligned");
  if (!(tol > 0.0)) return fail(MAGNUS_EINVAL, "magnus_expv_xxz_static: tol must be > 0");
  for (int k = 0; k < 2; k++)
    if (!(beta[k] == beta[k]) || beta[k] - beta[k] != 0.0)
      return fail(MAGNUS_EINVAL, "magnus_expv_xxz_static: beta not finite");

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64)
    return fail(MAGNUS_ECUDA, "magnus_expv_xxz_static: no current CUDA device");
  DeviceSetup S;
  {
    // First call on this device: resolve the scratch address and compute the Leja points into it.
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    DeviceSetup &s = g_setup[dev];
    if (!s.done) {
      void *ptr = nullptr;
      if (cudaGetSymbolAddress(&ptr, g_static_scratch) != cudaSuccess || !ptr)
        return fail(MAGNUS_ECUDA, "magnus_expv_xxz_static: cudaGetSymbolAddress failed");
      unsigned char *base = (unsigned char *)ptr;
      if (cudaDeviceGetAttribute(&s.num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
          persistent_max_blocks_per_sm(FAM_GENERIC, false, 0, &s.blocks_per_sm) != cudaSuccess)
        return fail(MAGNUS_ECUDA, "magnus_expv_xxz_static: device query failed");
      if (launch_leja_points((double *)(base + kOffXi), kStaticMmax, (double *)(base + kOffCand),
                             (unsigned *)(base + kOffCounter), stream) != cudaSuccess ||
          cudaStreamSynchronize(stream) != cudaSuccess)
        return fail(MAGNUS_ECUDA, "magnus_expv_xxz_static: Leja point set-up failed");
      s.base = base;
      s.done = true;
    }
    S = s;
  }
  unsigned char *base = S.base;
  const int64_t D = (int64_t)1 << nspins;
  Term *terms = (Term *)(base + kOffTerms);
  double *term_ab = (double *)(base + kOffTermAB);
  ExpRec *rec = (ExpRec *)(base + kOffRec);
  double2 *dd = (double2 *)(base + kOffDD);
  GridBar *bar = (GridBar *)(base + kOffBar);
  Counters *counters = (Counters *)(base + kOffCounters);

  Term xxz{}, field{};
  xxz.kind = MAGNUS_TERM_XXZ;
  xxz.nspins = nspins;
  xxz.delta = delta;
  for (int i = 0; i < nspins - 1; i++) xxz.J[i] = J[i];
  for (int i = 0; i < nspins; i++) xxz.hz[i] = hz[i];
  field.kind = MAGNUS_TERM_FIELD_X;
  field.nspins = nspins;

  const int maxg = std::min(kStaticMaxGrid, S.num_sms * std::max(1, S.blocks_per_sm));
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(maxg, (D + 31) / 32));
  const int gblk = (int)std::max<int64_t>(1, std::min<int64_t>(kStaticGershBlocks, (D + 255) / 256));

  cudaError_t e = cudaSuccess;
  k_static_init<<<1, 32, 0, stream>>>(xxz, field, terms, bar, counters);
  e = cudaGetLastError();
  for (int k = 0; k < 2 && e == cudaSuccess; k++)
    e = launch_gershgorin(terms + k, k == 0 ? xxz : field, D, (double *)(base + kOffGersh), gblk, term_ab + 2 * k,
                          stream);
  if (e == cudaSuccess)
    e = launch_exp_setup_beta(beta, 2, term_ab, (const double *)(base + kOffXi), kStaticMmax, 4.0, rec, dd, stream);
  if (e == cudaSuccess && out != v)
    e = cudaMemcpyAsync(out, v, sizeof(double2) * (size_t)D, cudaMemcpyDeviceToDevice, stream);
  if (e == cudaSuccess) {
    PersistArgs a{};
    a.dim = D;
    a.nvec = 1;
    a.nterms = 2;
    a.gv = grid;
    a.m_max = kStaticMmax;
    a.nexp = 1;
    a.tol_rel = tol;
    a.tol_abs = tol;
    a.terms = terms;
    a.recs = rec;
    a.dd = dd;
    a.xi = (const double *)(base + kOffXi);
    a.psi = (double2 *)out;
    a.alt = (double2 *)(base + kOffVec);
    a.w0 = (double2 *)(base + kOffVec + kVecBytes);
    a.w1 = (double2 *)(base + kOffVec + 2 * kVecBytes);
    a.u = nullptr;  // only the M4 commutator uses it
    a.partials = (double *)(base + kOffPartials);
    a.bar = bar;
    a.counters = counters;
    a.mlog = nullptr;
    a.mlog_cap = 0;
    a.spin_limit_ns = 4000000000LL;
    a.fam = FAM_GENERIC;  // the instantiation whose occupancy sized the grid (zfix stays 0: FP64 sums)
    e = launch_persistent(a, grid, persistent_block_size(), false, stream);
  }
  Counters c{};
  if (e == cudaSuccess) e = cudaMemcpyAsync(&c, counters, sizeof c, cudaMemcpyDeviceToHost, stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return fail(MAGNUS_ECUDA, cudaGetErrorString(e));
  if (c.status != MAGNUS_OK) {
    return fail((magnus_status)c.status, c.status == MAGNUS_ENOCONV ? "magnus_expv_xxz_static: Leja did not converge"
                                         : c.status == MAGNUS_ETIMEOUT ? "magnus_expv_xxz_static: barrier timed out"
                                                                       : "magnus_expv_xxz_static: non-finite norm");
  }
  return MAGNUS_OK;
}
