// Differentiation of the rule estimate over a frozen box list: the backward
// pass of the converged integral (the paper defines no derivative).
#pragma once
#include "pagani_eval.cuh"

namespace pg {

// -------------------------------------------------- gradient, thread per box
// d/dtheta of the basic-rule estimate summed over a fixed list of boxes (the
// leaf set of an integration), and the estimate itself, for theta = (p0_j,
// p1_j) of every axis.  One thread per box.
//
// For a product integrand f = prod_j phi_j(x_j), the box's basic-rule value
// V = sum_g w_g sum_{x in orbit g} f(x) is multilinear in the per-axis factor
// values t_j(c) = phi_j(x at code c): every rule point takes exactly one
// factor from each axis.  Summed over the +/- signs of an orbit, the factors
// of one non-centre radius enter only as s_j(r) = t_j(r+) + t_j(r-), so
//   V = w_0 P + sum_j Q_j (w_1 s_j(1) + w_2 s_j(2) + w_3 s_j(3))
//     + sum_{j<k} Q_jk (w_5 s_j(1) s_k(1) + w_6 (s_j(1) s_k(2) + s_j(2) s_k(1)))
//     + sum_{j<k<l} w_7 Q_jkl s_j(1) s_k(1) s_l(1) + w_8 prod_j s_j(0),
// with P the product of the centre factors and Q_... the same product
// without the named axes (the lambda_p orbit has zero basic weight).  These
// sums are coefficients of one polynomial, prod_j (t0_j + z s_j(1) +
// y s_j(2) + x s_j(3)), so prefix and suffix products of it give V and
// H_j(r) = dV/ds_j(r) in O(n) operations.  By the chain rule, with
// dt_j(c)/dtheta = t_j(c) dlog phi_j(x_c)/dtheta,
//   dV/dtheta_j = sum_{c != C0} dlog_j(c) t_j(c) H_j(r(c)) + dlog_j(C0) G_j(C0),
// where G_j(C0) = V - sum_r s_j(r) H_j(r) is the part of V whose points sit
// at the centre on axis j (V is linear in axis j's factors, one per point).
// The orbit's 2, 4 or 8 sign combinations, and the 2^n vertices, are never
// formed one by one.
//
// The chain-rule factors depend only on the axis interval, like the factor
// values: per interval, dlog_j(C0) and, per radius r, sum over its two signs
// of t_j(c) dlog_j(c) (kGradTerms values).  They are tabulated for every
// cached interval ahead of the gradient kernel and computed in place for
// deeper levels, by the same function.  Per thread in shared memory: the 9
// factor values used per axis (C0, r1+-, r2+-, r3+-, r0+-), read from the
// factor cache where the box's level on that axis is cached, and the 2n + 1
// sums: plain over up to kGradChunk boxes, then added into Neumaier pairs.
constexpr int kGradChunk = 8;

template <int N, int GT>
struct GradSmem {
  static constexpr int kTab = 9;           // factor values per axis
  static constexpr int kSums = 2 * N + 1;  // V, d/dp0_j, d/dp1_j
  static constexpr size_t bytes =
      ((size_t)kSums * (sizeof(NSum) + sizeof(double)) + (size_t)kTab * N * sizeof(double)) * GT;
};

__device__ __forceinline__ int grad_code(int slot) {  // compact table slot -> Code
  return slot < 7 ? slot : slot + 2;                  // 0..6 as is, 7, 8 -> kR0P, kR0M
}

// The chain-rule terms of axis j for the box [lo, lo + 2h) from its nine
// factor values t[slot * TS]: o[0], o[1] = dlog phi_j / d(p0_j, p1_j) at the
// centre; o[2 + 2i], o[3 + 2i] = the sum over the two signs of radius i (r1,
// r2, r3, r0) of t dlog phi_j / d(p0_j, p1_j).
template <class F, int TS>
__device__ __forceinline__ void grad_axis_terms(const EvalRule& R, const IntegrandParams& prm, int j, double lo,
                                                double h, const double* t, double* o) {
  {
    double d0, d1;
    F::dlog(prm, j, point_x(prm, j, lo + h, h, 0.0), t[0], d0, d1);
    o[0] = d0;
    o[1] = d1;
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    double e0 = 0.0, e1 = 0.0;
#pragma unroll
    for (int sg = 0; sg < 2; ++sg) {
      const int slot = 2 * i + 1 + sg;
      const double tc = t[slot * TS];
      double d0, d1;
      F::dlog(prm, j, point_x(prm, j, lo + h, h, code_offset(R, grad_code(slot))), tc, d0, d1);
      e0 = fma(d0, tc, e0);
      e1 = fma(d1, tc, e1);
    }
    o[2 + 2 * i] = e0;
    o[3 + 2 * i] = e1;
  }
}

// Tabulates the chain-rule terms of every cached interval (levels <= L),
// slot 2^l - 1 + k for [k 2^-l, (k+1) 2^-l), as the factor cache does.
template <class F, int N>
__global__ void __launch_bounds__(256) k_grad_terms(const EvalRule R, const GradArgs A) {
  const IntegrandParams& prm = *A.prm;
  const long long slots = (2LL << A.fcache_levels) - 1;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < (long long)N * slots;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long slot = idx % slots;
    const int j = (int)(idx / slots);
    const int L = 63 - __clzll(slot + 1);  // slot = 2^L - 1 + k
    const long long k = slot + 1 - (1LL << L);
    const double h = 0.5 * pow2_neg(L);
    const double lo = (double)k * pow2_neg(L);
    const typename F::Ax ax = F::axis(prm, j);
    double t[9], o[kGradTerms];
#pragma unroll
    for (int q = 0; q < 9; ++q) t[q] = F::factor(ax, point_x(prm, j, lo + h, h, code_offset(R, grad_code(q))));
    grad_axis_terms<F, 1>(R, prm, j, lo, h, t, o);
    double* dst = A.terms + ((size_t)j * kCacheSlots + slot) * kGradTerms;
#pragma unroll
    for (int q = 0; q < kGradTerms; ++q) dst[q] = o[q];
  }
}

template <class F, int N, int GT>
__global__ void __launch_bounds__(GT) k_gradient_box(const EvalRule R, const GradArgs A) {
  extern __shared__ __align__(16) unsigned char gsmem[];
  constexpr int K = GradSmem<N, GT>::kSums;
  NSum* acc = reinterpret_cast<NSum*>(gsmem);                           // [k][thread]
  double* part = reinterpret_cast<double*>(acc + K * GT) + threadIdx.x;  // [k], stride GT: plain chunk sums
  double* tab = part + K * GT;                                          // [slot][j], stride GT
#define PG_T(slot, j) tab[((slot) * N + (j)) * GT]
  const IntegrandParams& prm = *A.prm;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    acc[k * GT + threadIdx.x] = NSum{0.0, 0.0};
    part[k * GT] = 0.0;
  }
  const double w0 = R.w[kGenCentre][0], w1 = R.w[kGenL1][0], w2 = R.w[kGenL2][0], w3 = R.w[kGenL3][0];
  const double w5 = R.w[kGenL1L1][0], w6 = R.w[kGenL1L2][0], w7 = R.w[kGenL1L1L1][0], w8 = R.w[kGenL0All][0];
  const bool cached = A.fcache != nullptr && A.terms != nullptr;
  int chunk = 0;
  for (int64_t r = (int64_t)blockIdx.x * GT + threadIdx.x; r < A.m; r += (int64_t)gridDim.x * GT) {
    int L = 0;
    double s1[N], s2[N], s3[N], s0[N];
#pragma unroll
    for (int j = 0; j < N; ++j) {
      const double lo = A.lower[(size_t)j * A.m + r];
      const int lv = A.level[(size_t)j * A.m + r];
      L += lv;
      if (cached && lv <= A.fcache_levels) {  // same expression, same bits
        const double* src = A.fcache + ((size_t)j * kCacheSlots + ((1 << lv) - 1) + dyadic_index(lo, lv)) * kCodes;
#pragma unroll
        for (int slot = 0; slot < GradSmem<N, GT>::kTab; ++slot) PG_T(slot, j) = src[grad_code(slot)];
      } else {
        const double h = 0.5 * pow2_neg(lv);
        const typename F::Ax ax = F::axis(prm, j);
#pragma unroll
        for (int slot = 0; slot < GradSmem<N, GT>::kTab; ++slot)
          PG_T(slot, j) = F::factor(ax, point_x(prm, j, lo + h, h, code_offset(R, grad_code(slot))));
      }
      s1[j] = PG_T(1, j) + PG_T(2, j);
      s2[j] = PG_T(3, j) + PG_T(4, j);
      s3[j] = PG_T(5, j) + PG_T(6, j);
      s0[j] = PG_T(7, j) + PG_T(8, j);
    }
    // The centre, one-axis, pair and triple orbit sums are coefficients of
    // prod_j (t0_j + z s_j(1) + y s_j(2) + x s_j(3)): of 1, z, y, x, z^2,
    // zy, z^3.  Prefix products P_j (over the axes before j) keep the
    // coefficients of 1, z, y, z^2, and the full product also x, zy, z^3.
    double P1[N + 1], Pz[N + 1], Py[N + 1], Pzz[N + 1];
    double px = 0.0, pzy = 0.0, pzzz = 0.0;
    P1[0] = 1.0;
    Pz[0] = Py[0] = Pzz[0] = 0.0;
#pragma unroll
    for (int m = 0; m < N; ++m) {
      const double t0 = PG_T(0, m);
      px = fma(px, t0, P1[m] * s3[m]);
      pzy = fma(pzy, t0, fma(Pz[m], s2[m], Py[m] * s1[m]));
      pzzz = fma(pzzz, t0, Pzz[m] * s1[m]);
      P1[m + 1] = P1[m] * t0;
      Pz[m + 1] = fma(Pz[m], t0, P1[m] * s1[m]);
      Py[m + 1] = fma(Py[m], t0, P1[m] * s2[m]);
      Pzz[m + 1] = fma(Pzz[m], t0, Pz[m] * s1[m]);
    }
    // every axis at r0: w_8 prod_j s_j(0), and its leave-one-out products
    double H0[N];
    double V;
    {
      double run = w8;
#pragma unroll
      for (int m = 0; m < N; ++m) {
        H0[m] = run;
        run *= s0[m];
      }
      double sr = 1.0;
#pragma unroll
      for (int m = N - 1; m >= 0; --m) {
        H0[m] *= sr;
        sr *= s0[m];
      }
      V = fma(w0, P1[N], fma(w1, Pz[N], fma(w2, Py[N], fma(w3, px, fma(w5, Pzz[N], fma(w6, pzy, fma(w7, pzzz, run)))))));
    }
    // per axis, last to first with the suffix product Q (coefficients of 1,
    // z, y, z^2): the leave-one-out product L_j = P_j Q, then
    // H_j(r) = dV/ds_j(r), then the chain rule through the tabulated terms
    const double vol = pow2_neg(L) * prm.vol;
    part[0] = fma(vol, V, part[0]);
    double q1 = 1.0, qz = 0.0, qy = 0.0, qzz = 0.0;
#pragma unroll
    for (int j = N - 1; j >= 0; --j) {
      const double L1 = P1[j] * q1;
      const double Lz = fma(P1[j], qz, Pz[j] * q1);
      const double Ly = fma(P1[j], qy, Py[j] * q1);
      const double Lzz = fma(P1[j], qzz, fma(Pz[j], qz, Pzz[j] * q1));
      const double H1 = fma(w1, L1, fma(w5, Lz, fma(w6, Ly, w7 * Lzz)));
      const double H2 = fma(w2, L1, w6 * Lz);
      const double H3 = w3 * L1;
      {
        const double t0 = PG_T(0, j);
        const double nz = fma(qz, t0, q1 * s1[j]), ny = fma(qy, t0, q1 * s2[j]), nzz = fma(qzz, t0, qz * s1[j]);
        q1 *= t0;
        qz = nz;
        qy = ny;
        qzz = nzz;
      }
      const double lo = A.lower[(size_t)j * A.m + r];
      const int lv = A.level[(size_t)j * A.m + r];
      double o[kGradTerms];
      if (cached && lv <= A.fcache_levels) {
        const double* src =
            A.terms + ((size_t)j * kCacheSlots + ((1 << lv) - 1) + dyadic_index(lo, lv)) * kGradTerms;
#pragma unroll
        for (int q = 0; q < kGradTerms; ++q) o[q] = src[q];
      } else {
        grad_axis_terms<F, N * GT>(R, prm, j, lo, 0.5 * pow2_neg(lv), &PG_T(0, j), o);
      }
      // the part of V at the centre on axis j
      const double gc = V - fma(s1[j], H1, fma(s2[j], H2, fma(s3[j], H3, s0[j] * H0[j])));
      double g0 = o[0] * gc, g1 = o[1] * gc;
      g0 = fma(o[2], H1, g0);
      g1 = fma(o[3], H1, g1);
      g0 = fma(o[4], H2, g0);
      g1 = fma(o[5], H2, g1);
      g0 = fma(o[6], H3, g0);
      g1 = fma(o[7], H3, g1);
      g0 = fma(o[8], H0[j], g0);
      g1 = fma(o[9], H0[j], g1);
      part[(1 + j) * GT] = fma(vol, g0, part[(1 + j) * GT]);
      part[(1 + N + j) * GT] = fma(vol, g1, part[(1 + N + j) * GT]);
    }
    if (++chunk == kGradChunk) {  // plain over the chunk, compensated across chunks
      chunk = 0;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        NSum t = acc[k * GT + threadIdx.x];
        nadd(t, part[k * GT]);
        acc[k * GT + threadIdx.x] = t;
        part[k * GT] = 0.0;
      }
    }
  }
#pragma unroll
  for (int k = 0; k < K; ++k) {
    NSum t = acc[k * GT + threadIdx.x];
    nadd(t, part[k * GT]);
    acc[k * GT + threadIdx.x] = t;
  }
#undef PG_T
  // block, then grid reduction (fixed order)
  __syncthreads();
  NSum* red = acc;
  if (threadIdx.x < K) {
    NSum t = red[threadIdx.x * GT];
    for (int q = 1; q < GT; ++q) t = ncomb(t, red[threadIdx.x * GT + q]);
    A.part[((size_t)blockIdx.x * K + threadIdx.x) * 2] = t.s;
    A.part[((size_t)blockIdx.x * K + threadIdx.x) * 2 + 1] = t.c;
  }
  if (!last_block_arrived(A.ticket)) return;
  // K sums over the blocks: threads split the blocks of each sum, then fold
  __syncthreads();
  constexpr int PER = GT / K > 0 ? GT / K : 1;
  if (threadIdx.x < K * PER) {
    const int k = threadIdx.x / PER, part = threadIdx.x % PER;
    NSum t = {0.0, 0.0};
    for (unsigned b = part; b < gridDim.x; b += PER) {
      NSum q;
      q.s = A.part[((size_t)b * K + k) * 2];
      q.c = A.part[((size_t)b * K + k) * 2 + 1];
      t = ncomb(t, q);
    }
    red[threadIdx.x] = t;
  }
  __syncthreads();
  if (threadIdx.x < K) {
    NSum t = red[threadIdx.x * PER];
    for (int q = 1; q < PER; ++q) t = ncomb(t, red[threadIdx.x * PER + q]);
    A.out[threadIdx.x] = nval(t);
  }
}

// ---------------------------------------------------------------- launcher
template <class F, int N>
cudaError_t launch_grad(const EvalRule& R, const GradArgs& A, int grid, cudaStream_t st) {
  if constexpr (F::kHasGrad) {
    const size_t smem = GradSmem<N, kGradThreads>::bytes;
    static bool attr = false;
    if (!attr) {
      cudaFuncSetAttribute((const void*)&k_gradient_box<F, N, kGradThreads>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      attr = true;
    }
    if (A.terms != nullptr && A.fcache != nullptr) {
      const long long entries = (long long)N * ((2LL << A.fcache_levels) - 1);
      k_grad_terms<F, N><<<(int)((entries + 255) / 256), 256, 0, st>>>(R, A);
      const cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
    k_gradient_box<F, N, kGradThreads><<<grid, kGradThreads, smem, st>>>(R, A);
    return cudaGetLastError();
  } else {
    return cudaErrorNotSupported;
  }
}

}  // namespace pg
