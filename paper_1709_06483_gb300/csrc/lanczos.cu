// Lanczos enclosure of one stored term's spectrum (arXiv:1709.06483, Sec. 3: the Leja method needs
// an enclosure of the spectrum of the matrix; the Gershgorin enclosure is rigorous but wide).
// m steps of the Lanczos recurrence on H_k from a fixed pseudo-random start vector
//     w = H v_j;  al_j = Re <v_j, w>;  w -= al_j v_j + be_j v_{j-1};  be_{j+1} = |w|;  v_{j+1} = w / be_{j+1}
// (stopped at an invariant subspace), then the extreme eigenvalues theta of the tridiagonal matrix
// by Sturm bisection and the residual norms r = be_m |s_last| of their Ritz vectors by inverse
// iteration.  The enclosure is [theta_min - r_min - 0.01 W, theta_max + r_max + 0.01 W] intersected
// with the Gershgorin one (W = theta_max - theta_min).  Runs once per plan; every step is a kernel,
// the scalars stay on the device, the reductions are in a fixed order.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "magnus_internal.cuh"
#include "persist_common.cuh"
#include "rows.cuh"

namespace mg {
namespace {

constexpr int kLzBlock = 256;
constexpr int kLzGrid = 152 * 4;

struct LzState {
  int stopped;  // an invariant subspace was reached
  int mj;       // Lanczos steps taken
  double amax, bmax;
};

// SplitMix64 (Steele, Lea, Flood 2014), output c of the stream that starts at `seed`.
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t c) {
  uint64_t z = seed + (c + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ double unit_at(uint64_t seed, uint64_t c) {
  return (double)(splitmix64_at(seed, c) >> 11) * 0x1.0p-53;
}

__device__ __forceinline__ void block_partial(double x, double *part) {
  __shared__ double s[kLzBlock / 32];
  x = warp_sum(x);
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = x;
  __syncthreads();
  if (threadIdx.x == 0) {
    double y = 0.0;
    for (int w = 0; w < kLzBlock / 32; w++) y += s[w];
    part[blockIdx.x] = y;
  }
}

// v_i = (2 u_{2i} - 1) + i (2 u_{2i+1} - 1); partial sums of |v_i|^2
__global__ void k_lz_start(double2 *v, int64_t D, uint64_t seed, double *part) {
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < D; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 x = make_double2(2.0 * unit_at(seed, 2 * (uint64_t)i) - 1.0, 2.0 * unit_at(seed, 2 * (uint64_t)i + 1) - 1.0);
    v[i] = x;
    s += cabs2(x);
  }
  block_partial(s, part);
}

// out = sum of part[0..n) in a fixed order (one block)
__global__ void k_lz_reduce(const double *part, int n, double *out, int take_sqrt) {
  double y = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) y += part[i];
  __shared__ double s[kLzBlock / 32];
  y = warp_sum(y);
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = y;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kLzBlock / 32; w++) t += s[w];
    *out = take_sqrt ? sqrt(t) : t;
  }
}

__global__ void k_lz_scale(double2 *v, const double *norm, int64_t D, const LzState *st) {
  if (st->stopped) return;
  const double inv = 1.0 / *norm;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < D; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 x = v[i];
    v[i] = make_double2(x.x * inv, x.y * inv);
  }
}

// w = H v (CSR, matrix-free and transverse-field terms: one thread per row); partials of Re <v, w>
__global__ void k_lz_apply(const Term *tp, const double2 *v, double2 *w, int64_t D, double *part, const LzState *st) {
  if (st->stopped) return;
  const Term &t = *tp;
  double s = 0.0;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < D; r += (int64_t)gridDim.x * blockDim.x) {
    const double2 y = rows::term_row_generic(t, v, r);
    w[r] = y;
    const double2 x = v[r];
    s = fma(x.x, y.x, fma(x.y, y.y, s));
  }
  block_partial(s, part);
}

// w = H v for a dense term (one warp per row); partials of Re <v, w>
__global__ void k_lz_apply_dense(const Term *tp, const double2 *v, double2 *w, int64_t D, double *part,
                                 const LzState *st) {
  if (st->stopped) return;
  const Term &t = *tp;
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double s = 0.0;
  for (int64_t r = warp0; r < D; r += nw) {
    double2 acc = make_double2(0.0, 0.0);
    if (t.rs == 1 || t.real_valued) {
      for (int64_t j = lane; j < D; j += 32) acc = rfma(t.rv[(r * D + j) * t.rs], v[j], acc);
    } else {
      for (int64_t j = lane; j < D; j += 32) acc = cfma(t.val[r * D + j], v[j], acc);
    }
    acc.x = warp_sum(acc.x);
    acc.y = warp_sum(acc.y);
    if (lane == 0) {
      w[r] = acc;
      const double2 x = v[r];
      s = fma(x.x, acc.x, fma(x.y, acc.y, s));
    }
  }
  block_partial(s, part);
}

// w -= al_j v + be_j v_prev; partials of |w|^2
__global__ void k_lz_update(double2 *w, const double2 *v, const double2 *vp, const double *al, const double *be, int j,
                            int64_t D, double *part, const LzState *st) {
  if (st->stopped) return;
  const double a = al[j], b = be[j];
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < D; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 x = v[i], y = vp[i];
    double2 z = w[i];
    z.x -= fma(a, x.x, b * y.x);
    z.y -= fma(a, x.y, b * y.y);
    w[i] = z;
    s += cabs2(z);
  }
  block_partial(s, part);
}

// after step j: al[j] and be[j+1] are known; track the scale, detect an invariant subspace
__global__ void k_lz_step_end(double *al, double *be, int j, LzState *st) {
  if (st->stopped) return;
  st->mj = j + 1;
  st->amax = fmax(st->amax, fabs(al[j]));
  st->bmax = fmax(st->bmax, be[j + 1]);
  if (be[j + 1] <= 1e-12 * (st->amax + st->bmax)) {
    be[j + 1] = 0.0;
    st->stopped = 1;
  }
}

__device__ int sturm_count(const double *al, const double *be, int m, double x) {
  int cnt = 0;
  double q = 1.0;
  for (int i = 0; i < m; i++) {
    const double off = (i > 0) ? be[i] * be[i] / q : 0.0;
    q = al[i] - x - off;
    if (q == 0.0) q = -1e-300;
    if (q < 0.0) cnt++;
  }
  return cnt;
}

// idx-th smallest eigenvalue of the tridiagonal (diagonal al, off-diagonal be[1..m-1]) by bisection
__device__ double tridiag_eig(const double *al, const double *be, int m, int idx) {
  double lo = INFINITY, hi = -INFINITY;
  for (int i = 0; i < m; i++) {
    const double r = (i > 0 ? fabs(be[i]) : 0.0) + (i + 1 < m ? fabs(be[i + 1]) : 0.0);
    lo = fmin(lo, al[i] - r);
    hi = fmax(hi, al[i] + r);
  }
  for (int it = 0; it < 200; it++) {
    const double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (sturm_count(al, be, m, mid) > idx) hi = mid; else lo = mid;
  }
  return 0.5 * (lo + hi);
}

// |last component| of the unit eigenvector for theta: inverse iteration with a shift outside the
// spectrum (T - sig I definite: the tridiagonal elimination needs no pivoting); x, c, d: scratch [m]
__device__ double tridiag_last(const double *al, const double *be, int m, double sig, double *x, double *c, double *d) {
  for (int i = 0; i < m; i++) x[i] = 1.0;
  for (int it = 0; it < 3; it++) {
    double piv = al[0] - sig;
    c[0] = (m > 1) ? be[1] / piv : 0.0;
    d[0] = x[0] / piv;
    for (int i = 1; i < m; i++) {
      piv = (al[i] - sig) - be[i] * c[i - 1];
      c[i] = (i + 1 < m) ? be[i + 1] / piv : 0.0;
      d[i] = (x[i] - be[i] * d[i - 1]) / piv;
    }
    x[m - 1] = d[m - 1];
    for (int i = m - 2; i >= 0; i--) x[i] = d[i] - c[i] * x[i + 1];
    double n2 = 0.0;
    for (int i = 0; i < m; i++) n2 += x[i] * x[i];
    const double inv = 1.0 / sqrt(n2);
    for (int i = 0; i < m; i++) x[i] *= inv;
  }
  return fabs(x[m - 1]);
}

// ab: in the Gershgorin enclosure, out the intersection with the Lanczos enclosure (one thread)
__global__ void k_lz_finish(const double *al, const double *be, const LzState *st, double *scratch, double *ab) {
  const int m = st->mj;
  if (m < 1) return;
  const double tmin = tridiag_eig(al, be, m, 0), tmax = tridiag_eig(al, be, m, m - 1);
  const double W = tmax - tmin;
  const double eps = 1e-9 * (fabs(tmin) + fabs(tmax) + W + 1e-300);
  double rmin = 0.0, rmax = 0.0;
  if (be[m] > 0.0) {
    rmin = be[m] * tridiag_last(al, be, m, tmin - eps, scratch, scratch + m, scratch + 2 * m);
    rmax = be[m] * tridiag_last(al, be, m, tmax + eps, scratch, scratch + m, scratch + 2 * m);
  }
  ab[0] = fmax(ab[0], tmin - rmin - 0.01 * W);
  ab[1] = fmin(ab[1], tmax + rmax + 0.01 * W);
}

}  // namespace

cudaError_t lanczos_interval(const Term *t_dev, const Term &t_host, int64_t D, int m, double *ab_dev, cudaStream_t st) {
  if (m > D) m = (int)D;
  double2 *buf = nullptr;
  double *sc = nullptr;
  LzState *state = nullptr;
  // scratch: 3 vectors; part [kLzGrid]; al [m+1]; be [m+2]; norm; tridiagonal scratch [3m]
  cudaError_t e = cudaMalloc((void **)&buf, sizeof(double2) * 3 * (size_t)D);
  if (e == cudaSuccess) e = cudaMalloc((void **)&sc, sizeof(double) * (kLzGrid + (m + 1) + (m + 2) + 1 + 3 * m));
  if (e == cudaSuccess) e = cudaMalloc((void **)&state, sizeof(LzState));
  if (e == cudaSuccess) e = cudaMemsetAsync(sc, 0, sizeof(double) * (kLzGrid + (m + 1) + (m + 2) + 1 + 3 * m), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(state, 0, sizeof(LzState), st);
  double *part = sc, *al = sc + kLzGrid, *be = al + (m + 1), *nrm = be + (m + 2), *tri = nrm + 1;
  double2 *vp = buf, *v = buf + D, *w = buf + 2 * D;
  const bool dense = t_host.kind == MAGNUS_TERM_DENSE;
  if (e == cudaSuccess) {
    cudaMemsetAsync(vp, 0, sizeof(double2) * (size_t)D, st);
    k_lz_start<<<kLzGrid, kLzBlock, 0, st>>>(v, D, 1709064830ull, part);
    k_lz_reduce<<<1, kLzBlock, 0, st>>>(part, kLzGrid, nrm, 1);
    k_lz_scale<<<kLzGrid, kLzBlock, 0, st>>>(v, nrm, D, state);
    for (int j = 0; j < m; j++) {
      if (dense)
        k_lz_apply_dense<<<kLzGrid, kLzBlock, 0, st>>>(t_dev, v, w, D, part, state);
      else
        k_lz_apply<<<kLzGrid, kLzBlock, 0, st>>>(t_dev, v, w, D, part, state);
      k_lz_reduce<<<1, kLzBlock, 0, st>>>(part, kLzGrid, al + j, 0);
      k_lz_update<<<kLzGrid, kLzBlock, 0, st>>>(w, v, vp, al, be, j, D, part, state);
      k_lz_reduce<<<1, kLzBlock, 0, st>>>(part, kLzGrid, be + j + 1, 1);
      k_lz_step_end<<<1, 1, 0, st>>>(al, be, j, state);
      // v_{j+1} = w / be_{j+1} into the buffer of v_{j-1}
      cudaMemcpyAsync(vp, w, sizeof(double2) * (size_t)D, cudaMemcpyDeviceToDevice, st);
      k_lz_scale<<<kLzGrid, kLzBlock, 0, st>>>(vp, be + j + 1, D, state);
      double2 *t = vp; vp = v; v = t;
    }
    k_lz_finish<<<1, 1, 0, st>>>(al, be, state, tri, ab_dev);
    e = cudaGetLastError();
  }
  cudaError_t e2 = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = e2;
  cudaFree(buf);
  cudaFree(sc);
  cudaFree(state);
  return e;
}

}  // namespace mg
