// Adjoint of the commutator-free Magnus propagation (arXiv:1709.06483, Sec. 2, Methods Cf4, Cf4:3,
// M2; each exponential by the Leja recurrence of Sec. 3): the gradient of F = |<phi|psi(T)>|^2 with
// respect to the drive coefficients of one term H_kd.
//
// For the exponentials U_e = exp(Omega_e), Omega_e = -i K_e, applied in order e = 0..M-1:
//   dF/dc = 2 Re( conj(z) sum_e (d beta_{kd,e}/dc) <lambda_e, L(Omega_e, -i H_kd) v_e> ),
// z = <phi, psi(T)>, v_e the state before exponential e, lambda_e = U_{e+1}^H..U_{M-1}^H phi the
// costate after it.  L(Omega, E) v is the first block of exp([[Omega, E], [0, Omega]]) [0; v]; the
// block matrix has Omega's spectrum, so it reuses the exponential's enclosure, shift, scale and
// divided differences, with the recurrence run on stacked vectors (k_aug_persistent).  The costate
// goes backward with exp(+i K_e) = exp(-i(-K_e)): the same records with every weight negated and the
// phase conjugated (k_negate_records).
#include <math.h>

#include <algorithm>

#include "magnus_internal.cuh"
#include "persist_common.cuh"
#include "rows.cuh"

namespace mg {

namespace {

using namespace rows;

constexpr int kABlock = 256;

// ZF: fixed-point sums and products (as in the propagation kernel) on copies of both stacked
// vectors; their scales follow from bounds of each block's largest component, tracked with the norms.
template <int FAM, bool ZF>
__global__ void __launch_bounds__(kABlock, 2) k_aug_persistent(AugArgs a) {
  __shared__ Term sT[kMaxTerms];
  __shared__ ExpRec sR;
  __shared__ double s_jb[kMaxSpins], s_j2[kMaxSpins];
  __shared__ double s_red[2][kABlock / 32];
  __shared__ unsigned s_rmx[4][kABlock / 32];
  __shared__ double s_tot[6];  // two sums, then bounds of four maxima (a, b, p_a, p_b)
  __shared__ double s_wz[kMaxTerms];
  __shared__ long long s_cb[kMaxSpins], s_c2[kMaxSpins];
  __shared__ int s_cbe, s_c2e;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned G = gridDim.x;
  const int b = blockIdx.x;
  const int64_t D = a.dim;
  const int64_t rows_per = (((D + G - 1) / G) + 31) & ~(int64_t)31;
  const int64_t lo = min(D, (int64_t)b * rows_per), hi = min(D, lo + rows_per);
  const int nt = a.nterms;
  for (int i = tid; i < nt * (int)sizeof(Term) / 4; i += blockDim.x)
    reinterpret_cast<int *>(sT)[i] = reinterpret_cast<const int *>(a.terms)[i];
  if (tid == 0) sR = *a.rec;
  __syncthreads();
  Ctx cx{};
  cx.T = sT;
  cx.nt = nt;
  cx.n = sT[0].nspins;
  cx.lbits = a.lbits;
  cx.lomask = ((int64_t)1 << (a.lbits + 1)) - 1;
  cx.dlo = a.dlo;
  cx.dhi = a.dhi;
  cx.jb = s_jb;
  cx.j2 = s_j2;
  const ExpRec &R = sR;
  if (FAM == FAM_MF)
    for (int p = 1 + tid; p < cx.n; p += blockDim.x) {
      s_j2[p - 1] = 2.0 * sT[0].J[cx.n - p - 1];
      s_jb[p - 1] = s_j2[p - 1] * R.bg[0];
    }
  double opnorm = 0.0;  // ZF: sum_k |bg_k| ||H_k||_inf
  if (ZF) {
    __syncthreads();
    if (tid < nt) s_wz[tid] = R.bg[tid] * sT[tid].pval;
    for (int k = 0; k < nt; k++) opnorm = fma(fabs(R.bg[k]), sT[k].gnorm, opnorm);
    if (FAM == FAM_MF && tid == 0) {  // bond weights (scaled and unscaled) as 62-bit mantissas
      double w1 = 0.0, w2 = 0.0;
      for (int p = 0; p < cx.n - 1; p++) {
        w1 = fmax(w1, fabs(s_jb[p]));
        w2 = fmax(w2, fabs(s_j2[p]));
      }
      int E1 = 0, E2 = 0;
      if (w1 > 0.0) frexp(w1, &E1);
      if (w2 > 0.0) frexp(w2, &E2);
      E1 = max(-400, min(400, E1));
      E2 = max(-400, min(400, E2));
      for (int p = 0; p < cx.n - 1; p++) {
        s_cb[p] = llrint(ldexp(s_jb[p], 62 - E1));
        s_c2[p] = llrint(ldexp(s_j2[p], 62 - E2));
      }
      s_cbe = E1;
      s_c2e = E2;
    }
    __syncthreads();
    if (FAM == FAM_MF) {
      cx.cb = s_cb;
      cx.cbe = s_cbe;
      cx.c2 = s_c2;
      cx.c2e = s_c2e;
    }
  }
  unsigned it = 0;
  auto fail = [&](int status) {
    if (tid == 0) atomicCAS(&a.counters->status, 0, status);
  };
  // partial sums (and, ZF, maxima as abshi high words) of this block -> slot; barrier; every block
  // sums all slots in the same order
  auto reduce_all = [&](double x0, double x1, unsigned m0 = 0u, unsigned m1 = 0u, unsigned m2 = 0u,
                        unsigned m3 = 0u) -> bool {
    x0 = warp_sum(x0);
    x1 = warp_sum(x1);
    if (ZF) {
      m0 = __reduce_max_sync(kFull, m0);
      m1 = __reduce_max_sync(kFull, m1);
      m2 = __reduce_max_sync(kFull, m2);
      m3 = __reduce_max_sync(kFull, m3);
    }
    if (lane == 0) {
      s_red[0][warp] = x0;
      s_red[1][warp] = x1;
      if (ZF) { s_rmx[0][warp] = m0; s_rmx[1][warp] = m1; s_rmx[2][warp] = m2; s_rmx[3][warp] = m3; }
    }
    __syncthreads();
    double *slot = a.partials + (size_t)(it & 1u) * G * 6;
    if (tid == 0) {
      double y0 = 0.0, y1 = 0.0;
      unsigned n[4] = {0u, 0u, 0u, 0u};
      for (int w = 0; w < kABlock / 32; w++) {
        y0 += s_red[0][w];
        y1 += s_red[1][w];
        if (ZF)
          for (int q = 0; q < 4; q++) n[q] = max(n[q], s_rmx[q][w]);
      }
      slot[6 * b] = y0;
      slot[6 * b + 1] = y1;
      for (int q = 0; q < 4; q++) slot[6 * b + 2 + q] = __hiloint2double((int)n[q], 0);
    }
    if (!grid_barrier(a.bar, G, a.spin_limit_ns)) return false;
    if (warp == 0) {
      double y0 = 0.0, y1 = 0.0;
      unsigned n[4] = {0u, 0u, 0u, 0u};
      for (int q = lane; q < (int)G; q += 32) {
        y0 += slot[6 * q];
        y1 += slot[6 * q + 1];
        if (ZF)
          for (int c = 0; c < 4; c++) n[c] = max(n[c], (unsigned)__double2hiint(slot[6 * q + 2 + c]));
      }
      y0 = warp_sum(y0);
      y1 = warp_sum(y1);
      if (ZF)
        for (int c = 0; c < 4; c++) n[c] = __reduce_max_sync(kFull, n[c]);
      if (lane == 0) {
        s_tot[0] = y0;
        s_tot[1] = y1;
        for (int c = 0; c < 4; c++) s_tot[2 + c] = abshi_bound(n[c]);
      }
    }
    __syncthreads();
    it++;
    return true;
  };

  // [a; b] = [0; v]
  double s = 0.0;
  unsigned mv = 0u;
  for (int64_t r = lo + tid; r < hi; r += blockDim.x) {
    const double2 v = a.v[r];
    a.acur[r] = make_double2(0.0, 0.0);
    a.bcur[r] = v;
    s += cabs2(v);
    if (ZF) mv = max(mv, abshi(v));
  }
  if (!reduce_all(s, 0.0, 0u, mv)) { fail(MAGNUS_ETIMEOUT); return; }
  double vn = sqrt(s_tot[0]);
  double vma = 0.0, vmb = s_tot[3];  // ZF: bounds of the largest components of the substep input
  const double2 *d = a.dd;
  double2 *ca = a.acur, *cb = a.bcur, *na = a.anxt, *nb = a.bnxt;
  if (!(R.gamma > 0.0)) {
    // scalar K: exp(-i [[c, H], [0, c]]) [0; v] = e^{-ic} [-i H v; v]
    const double2 ph = d[0];
    for (int64_t r = lo + tid; r < hi; r += blockDim.x) {
      const double2 hv = Op<FAM>::term(cx, a.kd, cb, r);
      a.out_a[r] = cmul(ph, make_double2(hv.y, -hv.x));
    }
    return;
  }
  const double invg = 1.0 / R.gamma;
  const double2 d0 = d[0];
  const double zfac = a.zreal ? 1.0 : 2.0;
  for (int sub = 0; sub < R.s; sub++) {
    double ep = sqrt(cabs2(d0)) * vn, pn = vn;
    double ma = vma, mb = vmb, pma = vma, pmb = vmb;
    int zs_a = 0, zs_b = 0;
    if (ZF) {  // fixed-point copies of the substep input
      zs_a = fix_scale(vma, a.zhb);
      zs_b = fix_scale(vmb, a.zhb);
      for (int64_t r = lo + tid; r < hi; r += blockDim.x) {
        a.zca[r] = fix2(ca[r], zs_a);
        a.zcb[r] = fix2(cb[r], zs_b);
      }
      if (!grid_barrier(a.bar, G, a.spin_limit_ns)) { fail(MAGNUS_ETIMEOUT); return; }
    }
    bool done = false;
    for (int j = 1; j <= a.m_max; j++) {
      const double2 *sa = (j == 1) ? ca : (((j - 2) & 1) ? a.wa1 : a.wa0);
      const double2 *sb = (j == 1) ? cb : (((j - 2) & 1) ? a.wb1 : a.wb0);
      double2 *da = ((j - 1) & 1) ? a.wa1 : a.wa0;
      double2 *db = ((j - 1) & 1) ? a.wb1 : a.wb0;
      const double shift = R.cg + a.xi[j - 1];
      const double2 dj = d[j];
      double sw = 0.0, sp = 0.0;
      unsigned mya = 0u, myb = 0u, mpa = 0u, mpb = 0u;
      int ys_a = 0, ys_b = 0;
      if constexpr (ZF) {
        // |y_a| <= (||X - shift|| max|a| + ||H_kd|| max|b| / gamma) (x2 complex), |y_b| <= ||X - shift|| max|b|
        const double on = opnorm + fabs(shift);
        ys_a = fix_scale(zfac * (on * ma + invg * sT[a.kd].gnorm * mb) * (1.0 + 0x1p-20), a.zhb);
        ys_b = fix_scale(zfac * on * mb * (1.0 + 0x1p-20), a.zhb);
        const longlong2 *za = (j == 1) ? a.zca : (((j - 2) & 1) ? a.zwa1 : a.zwa0);
        const longlong2 *zb = (j == 1) ? a.zcb : (((j - 2) & 1) ? a.zwb1 : a.zwb0);
        longlong2 *zda = ((j - 1) & 1) ? a.zwa1 : a.zwa0;
        longlong2 *zdb = ((j - 1) & 1) ? a.zwb1 : a.zwb0;
        for (int64_t r = lo + tid; r < hi; r += blockDim.x) {
          double2 xa, xb;
          double2 ya = Op<FAM>::combo_z(cx, R, s_wz, shift, sa, za, zs_a, r, xa);
          ya = rfma(invg, Op<FAM>::term_z(cx, a.kd, sb, zb, zs_b, r), ya);
          const double2 yb = Op<FAM>::combo_z(cx, R, s_wz, shift, sb, zb, zs_b, r, xb);
          da[r] = ya;
          db[r] = yb;
          zda[r] = fix2(ya, ys_a);
          zdb[r] = fix2(yb, ys_b);
          double2 pa = (j == 1) ? cmul(d0, xa) : na[r];
          double2 pb = (j == 1) ? cmul(d0, xb) : nb[r];
          pa = cfma(dj, ya, pa);
          pb = cfma(dj, yb, pb);
          na[r] = pa;
          nb[r] = pb;
          sw += cabs2(ya) + cabs2(yb);
          sp += cabs2(pa) + cabs2(pb);
          mya = max(mya, abshi(ya));
          myb = max(myb, abshi(yb));
          mpa = max(mpa, abshi(pa));
          mpb = max(mpb, abshi(pb));
        }
      } else {
        for (int64_t r = lo + tid; r < hi; r += blockDim.x) {
          double2 xa, xb;
          double2 ya = Op<FAM>::combo(cx, R, shift, sa, r, xa);
          ya = rfma(invg, Op<FAM>::term(cx, a.kd, sb, r), ya);
          const double2 yb = Op<FAM>::combo(cx, R, shift, sb, r, xb);
          da[r] = ya;
          db[r] = yb;
          double2 pa = (j == 1) ? cmul(d0, xa) : na[r];
          double2 pb = (j == 1) ? cmul(d0, xb) : nb[r];
          pa = cfma(dj, ya, pa);
          pb = cfma(dj, yb, pb);
          na[r] = pa;
          nb[r] = pb;
          sw += cabs2(ya) + cabs2(yb);
          sp += cabs2(pa) + cabs2(pb);
        }
      }
      if (!reduce_all(sw, sp, mya, myb, mpa, mpb)) { fail(MAGNUS_ETIMEOUT); return; }
      zs_a = ys_a;
      zs_b = ys_b;
      ma = s_tot[2];
      mb = s_tot[3];
      pma = s_tot[4];
      pmb = s_tot[5];
      const double ej = sqrt(cabs2(dj)) * sqrt(s_tot[0]);
      pn = sqrt(s_tot[1]);
      if (!isfinite(ej) || !isfinite(pn)) { fail(MAGNUS_ENONFINITE); return; }
      if (ej + ep <= a.tol_abs + a.tol_rel * pn) {
        done = true;
        if (b == 0 && tid == 0) {
          atomicAdd((unsigned long long *)&a.counters->n_matvec, (unsigned long long)j);
          atomicMax(&a.counters->max_m, j);
        }
        break;
      }
      ep = ej;
    }
    if (!done) { fail(MAGNUS_ENOCONV); return; }
    vn = pn;
    vma = pma;
    vmb = pmb;
    double2 *t = ca; ca = na; na = t;
    t = cb; cb = nb; nb = t;
  }
  for (int64_t r = lo + tid; r < hi; r += blockDim.x) a.out_a[r] = ca[r];
}

// rec' for exp(+iK) from rec for exp(-iK): weights, shift and centre negated, enclosure mirrored,
// divided differences with the conjugate phase (dd'_j = e^{2ic/s} dd_j).
__global__ void k_negate_records(const ExpRec *in, const double2 *din, ExpRec *out, double2 *dout, int64_t nexp,
                                 int m_max) {
  for (int64_t e = blockIdx.x; e < nexp; e += gridDim.x) {
    const ExpRec R = in[e];
    const double ang = 2.0 * R.c / R.s;
    const double2 ph = make_double2(cos(ang), sin(ang));
    for (int j = threadIdx.x; j <= m_max; j += blockDim.x)
      dout[e * (int64_t)(m_max + 1) + j] = cmul(ph, din[e * (int64_t)(m_max + 1) + j]);
    if (threadIdx.x == 0) {
      ExpRec Q = R;
      for (int k = 0; k < kMaxTerms; k++) Q.bg[k] = -R.bg[k];
      for (int k = 0; k < kMaxPairs; k++) Q.kg[k] = -R.kg[k];
      Q.cg = -R.cg;
      Q.c = -R.c;
      Q.a = -R.b;
      Q.b = -R.a;
      out[e] = Q;
    }
  }
}

// out = <x, y> = sum conj(x_i) y_i, one block, fixed order.
__global__ void k_dot(const double2 *x, const double2 *y, int64_t n, double2 *out) {
  __shared__ double sr[32], si[32];
  double re = 0.0, im = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double2 a = x[i], b = y[i];
    re = fma(a.x, b.x, fma(a.y, b.y, re));
    im = fma(a.x, b.y, fma(-a.y, b.x, im));
  }
  re = warp_sum(re);
  im = warp_sum(im);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { sr[w] = re; si[w] = im; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double R = 0.0, I = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); q++) { R += sr[q]; I += si[q]; }
    *out = make_double2(R, I);
  }
}

__device__ double drive_basis(const Coeff &c, int q, double t) {
  if (q == 0) return 1.0;
  const int m = q - 1;
  if (m < c.nmodes) return cos(c.om[m] * t);
  return sin(c.om[m - c.nmodes] * t);
}

// grad[q] = 2 Re(conj(z) sum_e (d beta_{kd,e} / d coef_q) G_e); one warp per coefficient q
// (q = 0: a0, 1..nmodes: ac, nmodes+1..2 nmodes: as).
__global__ void k_adjoint_contract(const double2 *G, const double2 *z, const Coeff *coeff, int variant, double t0,
                                   double h, int64_t nsteps, double *grad, int ng) {
  const int q = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (q >= ng) return;
  const Coeff &C = *coeff;
  const double r3 = sqrt(3.0), r15 = sqrt(15.0);
  double cn[3], w[3][3];
  int ns = 1, J = 1;
  if (variant == MAGNUS_CF4) {
    const double a1 = (3.0 - 2.0 * r3) / 12.0, a2 = (3.0 + 2.0 * r3) / 12.0;
    ns = 2; J = 2;
    cn[0] = 0.5 - r3 / 6.0; cn[1] = 0.5 + r3 / 6.0;
    w[0][0] = a2; w[0][1] = a1; w[1][0] = a1; w[1][1] = a2;
  } else if (variant == MAGNUS_CF4_3) {
    const double al[3][3] = {{37.0 / 240.0 - 10.0 * r15 / 261.0, -1.0 / 30.0, 37.0 / 240.0 + 10.0 * r15 / 261.0},
                             {-11.0 / 360.0, 23.0 / 45.0, -11.0 / 360.0},
                             {37.0 / 240.0 + 10.0 * r15 / 261.0, -1.0 / 30.0, 37.0 / 240.0 - 10.0 * r15 / 261.0}};
    ns = 3; J = 3;
    cn[0] = 0.5 - r15 / 10.0; cn[1] = 0.5; cn[2] = 0.5 + r15 / 10.0;
    for (int s = 0; s < 3; s++)
      for (int j = 0; j < 3; j++) w[s][j] = al[2 - s][j];
  } else {
    ns = 1; J = 1;
    cn[0] = 0.5;
    w[0][0] = 1.0;
  }
  double re = 0.0, im = 0.0;
  const int64_t nexp = nsteps * ns;
  for (int64_t e = lane; e < nexp; e += 32) {
    const int64_t n = e / ns;
    const int s = (int)(e % ns);
    const double tn = t0 + (double)n * h;
    double db = 0.0;
    for (int j = 0; j < J; j++) db += w[s][j] * drive_basis(C, q, tn + cn[j] * h);
    db *= h;
    re = fma(db, G[e].x, re);
    im = fma(db, G[e].y, im);
  }
  re = warp_sum(re);
  im = warp_sum(im);
  if (lane == 0) {
    const double2 zz = *z;
    grad[q] = 2.0 * (zz.x * re + zz.y * im);  // Re(conj(z) (re + i im))
  }
}

const void *aug_kernel(int fam, bool zf) {
  if (zf && fam == FAM_CSR) return (const void *)k_aug_persistent<FAM_CSR, true>;
  if (zf && fam == FAM_MF) return (const void *)k_aug_persistent<FAM_MF, true>;
  switch (fam) {
    case FAM_CSR: return (const void *)k_aug_persistent<FAM_CSR, false>;
    case FAM_MF: return (const void *)k_aug_persistent<FAM_MF, false>;
    default: return (const void *)k_aug_persistent<FAM_GENERIC, false>;
  }
}

}  // namespace

int aug_block_size() { return kABlock; }

cudaError_t aug_max_blocks_per_sm(int *n) {
  int best = 1 << 30;
  for (int fam = 0; fam < 3; fam++)
    for (int zf = 0; zf < 2; zf++) {
      int k = 0;
      cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&k, aug_kernel(fam, zf != 0), kABlock, 0);
      if (e != cudaSuccess) return e;
      best = k < best ? k : best;
    }
  *n = best;
  return cudaSuccess;
}

cudaError_t launch_aug_persistent(const AugArgs &a, int grid, cudaStream_t st) {
  AugArgs copy = a;
  void *args[] = {&copy};
  const bool zf = a.zfix && (a.fam == FAM_CSR || a.fam == FAM_MF);
  return cudaLaunchCooperativeKernel(aug_kernel(a.fam, zf), dim3(grid), dim3(kABlock), args, 0, st);
}

cudaError_t launch_negate_records(const ExpRec *in, const double2 *din, ExpRec *out, double2 *dout, int64_t nexp,
                                  int m_max, cudaStream_t st) {
  k_negate_records<<<(unsigned)std::min<int64_t>(nexp, 4096), 128, 0, st>>>(in, din, out, dout, nexp, m_max);
  return cudaGetLastError();
}

cudaError_t launch_dot(const double2 *x, const double2 *y, int64_t n, double2 *out, cudaStream_t st) {
  k_dot<<<1, 1024, 0, st>>>(x, y, n, out);
  return cudaGetLastError();
}

cudaError_t launch_adjoint_contract(const double2 *G, const double2 *z, const Coeff *coeff, int variant, double t0,
                                    double h, int64_t nsteps, double *grad, int ng, cudaStream_t st) {
  const int warps = 4;
  k_adjoint_contract<<<(ng + warps - 1) / warps, 32 * warps, 0, st>>>(G, z, coeff, variant, t0, h, nsteps, grad, ng);
  return cudaGetLastError();
}

}  // namespace mg
