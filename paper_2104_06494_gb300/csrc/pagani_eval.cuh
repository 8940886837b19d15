// Evaluate (Algorithm 2, Sec. 3.2): the degree-9 rule sum, the four null-rule
// values, the fourth-difference split axis, and, in the loop kernel, the
// two-level error, Rel-Err-Classify and the block partial sums of V and E.
//
// GB300 mapping.  FP64 issue rate is the bound (about 2 FMA/clk/SM), so the
// kernel spends FP64 instructions only where the arithmetic needs them:
//  * one thread evaluates one sibling pair (regions 2p and 2p+1).  The two
//    boxes differ along one axis, so the per-axis factor table (11 coordinate
//    codes x n axes, in shared memory) is built once and patched on one axis;
//  * each rule point's value is the product (or sum, for the corner peak) of
//    its per-axis factors, formed from shared prefix/suffix partial products
//    so a point costs one or two FP64 multiplies instead of n;
//  * the nine generator sums are accumulated per thread and weighted once
//    per region (rule and null rules);
//  * index arithmetic, table addressing and the rest run on the integer pipes.
#pragma once
#include <cstdint>

#include "pagani_device.cuh"

// Minimum resident blocks per SM requested for the Evaluate kernels (a
// register budget: 1 lets them use up to 255 registers, 3 caps them near
// 168 for 12 warps per SM).  Set at build time with -DPAGANI_EVAL_MINB=k.
#ifndef PAGANI_EVAL_MINB
#define PAGANI_EVAL_MINB 1
#endif

namespace pg {

// ------------------------------------------------------------------ families
// A family supplies: the element type T of its per-axis factors, the monoid
// (mul), the value of f at a point from its last two factors (last), the
// starting element (base), and the per-axis factor at coordinate x.

struct RealProduct {
  typedef double T;
  // S + f(point) where f(point) = a b: one FMA
  __device__ static __forceinline__ double acc(double S, T a, T b) { return fma(a, b, S); }
  static constexpr bool kUnitBounded = false;  // positive values: |S_g| = sum |f|
  static constexpr bool kHasGrad = true;        // f = prod_j phi_j(x_j; p0_j, p1_j), phi > 0
  // split-axis fourth difference at the rule's inner and outer radius (smooth
  // integrands); false: at its two inner radii (kinks, jumps)
  static constexpr bool kOuterSplit = true;
  __device__ static __forceinline__ T mul(T a, T b) { return a * b; }
  __device__ static __forceinline__ double last(T a, T b) { return a * b; }
  __device__ static __forceinline__ double val(T a) { return a; }
};

struct ProductPeak : RealProduct {  // prod_j 1/(c_j^-2 + (x_j - w_j)^2)
  static constexpr int kFamily = kFamProductPeak;
  struct Ax { double cm2, w; };
  __device__ static __forceinline__ Ax axis(const IntegrandParams& p, int j) {
    Ax a;
    a.cm2 = 1.0 / (p.p0[j] * p.p0[j]);
    a.w = p.p1[j];
    return a;
  }
  __device__ static __forceinline__ T base(const IntegrandParams&) { return 1.0; }
  __device__ static __forceinline__ T factor(const Ax& a, double x) {
    double t = x - a.w;
    return 1.0 / fma(t, t, a.cm2);
  }
  // d log phi / d c and d log phi / d w at x (phi = 1/(c^-2 + t^2))
  __device__ static __forceinline__ void dlog(const IntegrandParams& p, int j, double x, double phi, double& d0,
                                              double& d1) {
    const double c = p.p0[j], t = x - p.p1[j];
    d0 = 2.0 * phi / (c * c * c);
    d1 = 2.0 * t * phi;
  }
};

struct Gaussian : RealProduct {  // exp(-sum_j a_j^2 (x_j - w_j)^2)
  static constexpr int kFamily = kFamGaussian;
  struct Ax { double a, w; };
  __device__ static __forceinline__ Ax axis(const IntegrandParams& p, int j) {
    Ax a;
    a.a = p.p0[j];
    a.w = p.p1[j];
    return a;
  }
  __device__ static __forceinline__ T base(const IntegrandParams&) { return 1.0; }
  __device__ static __forceinline__ T factor(const Ax& a, double x) {
    double u = a.a * (x - a.w);
    return exp(-(u * u));
  }
  // d log phi / d a = -2 a t^2, d log phi / d w = 2 a^2 t (t = x - w)
  __device__ static __forceinline__ void dlog(const IntegrandParams& p, int j, double x, double, double& d0,
                                              double& d1) {
    const double a = p.p0[j], t = x - p.p1[j];
    d0 = -2.0 * a * t * t;
    d1 = 2.0 * a * a * t;
  }
};

struct C0Fam : RealProduct {  // exp(-sum_j a_j |x_j - w_j|)
  static constexpr bool kOuterSplit = false;  // kinks
  static constexpr int kFamily = kFamC0;
  struct Ax { double a, w; };
  __device__ static __forceinline__ Ax axis(const IntegrandParams& p, int j) {
    Ax a;
    a.a = p.p0[j];
    a.w = p.p1[j];
    return a;
  }
  __device__ static __forceinline__ T base(const IntegrandParams&) { return 1.0; }
  __device__ static __forceinline__ T factor(const Ax& a, double x) { return exp(-(a.a * fabs(x - a.w))); }
  // d log phi / d a = -|t|, d log phi / d w = a sgn(t) (t = x - w)
  __device__ static __forceinline__ void dlog(const IntegrandParams& p, int j, double x, double, double& d0,
                                              double& d1) {
    const double a = p.p0[j], t = x - p.p1[j];
    d0 = -fabs(t);
    d1 = t > 0.0 ? a : (t < 0.0 ? -a : 0.0);
  }
};

struct Oscillatory {  // cos(2 pi u + sum_j a_j x_j) = Re[e^{2 pi i u} prod_j e^{i a_j x_j}]
  static constexpr int kFamily = kFamOscillatory;
  static constexpr bool kUnitBounded = true;  // signed values with |f| <= 1
  static constexpr bool kHasGrad = false;
  static constexpr bool kOuterSplit = true;
  typedef double2 T;
  struct Ax { double a; };
  __device__ static __forceinline__ T mul(T a, T b) {
    T r;
    r.x = fma(a.x, b.x, -(a.y * b.y));
    r.y = fma(a.x, b.y, a.y * b.x);
    return r;
  }
  __device__ static __forceinline__ double last(T a, T b) { return fma(a.x, b.x, -(a.y * b.y)); }
  __device__ static __forceinline__ double acc(double S, T a, T b) { return fma(a.x, b.x, fma(-a.y, b.y, S)); }
  __device__ static __forceinline__ double val(T a) { return a.x; }
  __device__ static __forceinline__ Ax axis(const IntegrandParams& p, int j) {
    Ax a;
    a.a = p.p0[j];
    return a;
  }
  __device__ static __forceinline__ T base(const IntegrandParams& p) {
    T z;
    sincospi(2.0 * p.u, &z.y, &z.x);
    return z;
  }
  __device__ static __forceinline__ T factor(const Ax& a, double x) {
    T z;
    sincos(a.a * x, &z.y, &z.x);
    return z;
  }
};

template <int N>
struct CornerPeak {  // (1 + sum_j a_j x_j)^-(N+1): per-axis terms add up
  static constexpr int kFamily = kFamCornerPeak;
  static constexpr bool kUnitBounded = false;
  static constexpr bool kHasGrad = false;
  static constexpr bool kOuterSplit = true;
  typedef double T;
  struct Ax { double a; };
  __device__ static __forceinline__ T mul(T a, T b) { return a + b; }
  __device__ static __forceinline__ double outer(double s) {
    double r = 1.0 / s;
    double y = 1.0;
    double pw = r;
    // r^(N+1) by binary powering (exponent known at compile time)
#pragma unroll
    for (int e = N + 1; e > 0; e >>= 1) {
      if (e & 1) y *= pw;
      if (e > 1) pw *= pw;
    }
    return y;
  }
  __device__ static __forceinline__ double last(T a, T b) { return outer(a + b); }
  __device__ static __forceinline__ double acc(double S, T a, T b) { return S + outer(a + b); }
  __device__ static __forceinline__ double val(T a) { return outer(a); }
  __device__ static __forceinline__ Ax axis(const IntegrandParams& p, int j) {
    Ax a;
    a.a = p.p0[j];
    return a;
  }
  __device__ static __forceinline__ T base(const IntegrandParams&) { return 1.0; }
  __device__ static __forceinline__ T factor(const Ax& a, double x) { return a.a * x; }
};

struct Discontinuous : RealProduct {  // prod_j exp(a_j x_j) [x_j < w_j] (Genz discontinuous)
  static constexpr int kFamily = kFamDiscontinuous;
  static constexpr bool kHasGrad = false;  // not differentiable in w
  static constexpr bool kOuterSplit = false;  // jumps
  struct Ax { double a, w; };
  __device__ static __forceinline__ Ax axis(const IntegrandParams& p, int j) {
    Ax a;
    a.a = p.p0[j];
    a.w = p.p1[j];
    return a;
  }
  __device__ static __forceinline__ T base(const IntegrandParams&) { return 1.0; }
  __device__ static __forceinline__ T factor(const Ax& a, double x) { return x < a.w ? exp(a.a * x) : 0.0; }
  __device__ static __forceinline__ void dlog(const IntegrandParams&, int, double, double, double& d0, double& d1) {
    d0 = d1 = 0.0;
  }
};

// (sum_j x_j^2)^p, p >= 0: per-axis terms x_j^2 add up.  The element type
// carries the exponent next to the partial sum, so the point formulas see it.
struct BoxPower {
  static constexpr int kFamily = kFamBoxPower;
  static constexpr bool kUnitBounded = false;
  static constexpr bool kHasGrad = false;
  static constexpr bool kOuterSplit = true;
  typedef double2 T;  // (partial sum, exponent)
  struct Ax { double p; };
  // out of line: inlined into every unrolled rule point its loop, square root
  // and pow would multiply the kernel's code
  __device__ static __noinline__ double outer(double s, double p) {
    const double q = 2.0 * p;
    if (q == rint(q) && p < 64.0) {  // integer or half-integer power
      int k = (int)p;
      double r = 1.0, b = s;
      while (k > 0) {
        if (k & 1) r *= b;
        b *= b;
        k >>= 1;
      }
      return (q - 2.0 * (double)(int)p) != 0.0 ? r * sqrt(s) : r;
    }
    return pow(s, p);
  }
  __device__ static __forceinline__ T mul(T a, T b) { return make_double2(a.x + b.x, a.y); }
  __device__ static __forceinline__ double last(T a, T b) { return outer(a.x + b.x, a.y); }
  __device__ static __forceinline__ double acc(double S, T a, T b) { return S + outer(a.x + b.x, a.y); }
  __device__ static __forceinline__ double val(T a) { return outer(a.x, a.y); }
  __device__ static __forceinline__ Ax axis(const IntegrandParams& p, int) {
    Ax a;
    a.p = p.u;
    return a;
  }
  __device__ static __forceinline__ T base(const IntegrandParams& p) { return make_double2(0.0, p.u); }
  __device__ static __forceinline__ T factor(const Ax& a, double x) { return make_double2(x * x, a.p); }
  __device__ static __forceinline__ void dlog(const IntegrandParams&, int, double, double, double& d0, double& d1) {
    d0 = d1 = 0.0;
  }
};

// Offset g of a coordinate code on [-1, 1] (radius order: l1, l2, l3, lp, l0).
__device__ __forceinline__ double code_offset(const EvalRule& R, int code) {
  if (code == kC0) return 0.0;
  double r = R.radius[(code - 1) >> 1];
  return (code & 1) ? r : -r;
}

// Coordinate on axis j of the rule point with offset g in the box of centre
// c and half-width h (unit-cube coordinates), mapped onto the integration
// bounds: lo_j + len_j (c + h g).  Every path (tables, cache, gradient) forms
// it with this one expression; for the unit cube it is c + h g exactly.
__device__ __forceinline__ double point_x(const IntegrandParams& p, int j, double c, double h, double g) {
  return fma(p.len[j], fma(h, g, c), p.lo[j]);
}

// Build the 11 factor entries of one axis (centre c, half-width h).
template <class F, int N, int THREADS>
__device__ __forceinline__ void build_axis(typename F::T* tab, const EvalRule& R, const IntegrandParams& prm,
                                           double c, double h, int j) {
  const typename F::Ax ax = F::axis(prm, j);
#pragma unroll
  for (int code = 0; code < kCodes; ++code)
    tab[(code * N + j) * THREADS] = F::factor(ax, point_x(prm, j, c, h, code_offset(R, code)));
}

// k of a dyadic lower bound k 2^-level, from the IEEE fields (integer ops).
__device__ __forceinline__ long long dyadic_index(double lower, int level) {
  const long long bits = __double_as_longlong(lower);
  if (bits == 0) return 0;
  const int e = (int)((bits >> 52) & 0x7ff) - 1023;
  const long long mant = (bits & ((1LL << 52) - 1)) | (1LL << 52);
  const int shift = e + level - 52;
  return shift >= 0 ? (mant << shift) : (mant >> (-shift));
}

// Table entries of axis j for the box [lo, lo + 2^-lv): copied from the
// per-axis factor cache when the level is cached, computed otherwise.  The
// cache holds the same expression of the same arguments, so both give the
// same bits.
template <class F, int N, int THREADS, int SLOTS = kCacheSlots>
__device__ __forceinline__ void axis_entries(typename F::T* tab, const EvalRule& R, const IntegrandParams& prm,
                                             const typename F::T* __restrict__ cache, int cache_levels, double lo,
                                             int lv, int j) {
  if (cache != nullptr && lv <= cache_levels) {
    const typename F::T* src = cache + ((size_t)j * SLOTS + ((1 << lv) - 1) + dyadic_index(lo, lv)) * kCodes;
#pragma unroll
    for (int code = 0; code < kCodes; ++code) tab[(code * N + j) * THREADS] = src[code];
  } else {
    const double h = 0.5 * pow2_neg(lv);
    const typename F::Ax ax = F::axis(prm, j);
#pragma unroll
    for (int code = 0; code < kCodes; ++code)
      tab[(code * N + j) * THREADS] = F::factor(ax, point_x(prm, j, lo + h, h, code_offset(R, code)));
  }
}

// The fourth difference's weight q = (a / b)^2 for the radii the family's
// axis choice uses (see rule_sums).
template <class F, int DEG>
__device__ __forceinline__ double split_q(const EvalRule& R) {
  return (DEG == 9 && F::kOuterSplit) ? R.q_outer : R.q;
}

// The nine generator sums S[g] = sum over the orbit of g of f, and the
// fourth differences D[j], for one region whose factor table is `tab`.
// DEG 9: every orbit of the degree-9 rule.  DEG 7: the Genz-Malik rule's
// orbits only (centre, one axis at the lp and l2 slots, pairs at l1, the
// vertices); the other sums stay zero.
template <class F, int N, int THREADS, int DEG = 9>
__device__ __forceinline__ void rule_sums(const typename F::T* __restrict__ tab, typename F::T base, double q,
                                          double (&S)[kNumGen], double (&D)[N]) {
  typedef typename F::T T;
#define PG_TB(code, j) tab[((code) * N + (j)) * THREADS]
  // prefix products pre[j] = base * prod_{m<j} T0_m, suffix suf[j] = prod_{m>=j} T0_m
  T pre[N + 1];
  T suf[N + 1];
  pre[0] = base;
#pragma unroll
  for (int j = 0; j < N; ++j) pre[j + 1] = F::mul(pre[j], PG_TB(kC0, j));
  suf[N - 1] = PG_TB(kC0, N - 1);
#pragma unroll
  for (int j = N - 2; j >= 1; --j) suf[j] = F::mul(PG_TB(kC0, j), suf[j + 1]);

  const double f0 = F::val(pre[N]);
  S[kGenCentre] = f0;
#pragma unroll
  for (int g = 1; g < kNumGen; ++g) S[g] = 0.0;

  // one-axis generators and the fourth differences.  The difference takes
  // its points at two radii a < b (split_slots): for the degree-9 rule the
  // l2 and l1 slots on smooth families, the lp and l2 slots on families
  // with kinks or jumps; for the degree-7 one the lp and l2 slots
  // (sqrt(9/70), sqrt(9/10)).  Those two orbits enter it through their pair
  // sums (and, for signed families, its noise floor through their
  // magnitudes); the other one-axis orbits go straight into their sums.
  constexpr bool kOut = DEG == 9 && F::kOuterSplit;
  constexpr int kInP = kOut ? kR2P : kRpP, kInM = kOut ? kR2M : kRpM;
  constexpr int kOutP = kOut ? kR1P : kR2P, kOutM = kOut ? kR1M : kR2M;
#pragma unroll
  for (int j = 0; j < N; ++j) {
    T Q = (j == N - 1) ? pre[N - 1] : F::mul(pre[j], suf[j + 1]);
    double pin = 0.0, min_ = 0.0, pout = 0.0, mout = 0.0, si, so;
    if constexpr (F::kUnitBounded) {
      pin = F::last(Q, PG_TB(kInP, j));
      min_ = F::last(Q, PG_TB(kInM, j));
      pout = F::last(Q, PG_TB(kOutP, j));
      mout = F::last(Q, PG_TB(kOutM, j));
      si = pin + min_;
      so = pout + mout;
    } else {
      si = F::acc(F::last(Q, PG_TB(kInM, j)), Q, PG_TB(kInP, j));
      so = F::acc(F::last(Q, PG_TB(kOutM, j)), Q, PG_TB(kOutP, j));
    }
    if constexpr (kOut) {
      S[kGenL1] += so;
      S[kGenL2] += si;
      S[kGenLp] = F::acc(F::acc(S[kGenLp], Q, PG_TB(kRpP, j)), Q, PG_TB(kRpM, j));
    } else {
      if constexpr (DEG == 9) S[kGenL1] = F::acc(F::acc(S[kGenL1], Q, PG_TB(kR1P, j)), Q, PG_TB(kR1M, j));
      S[kGenLp] += si;
      S[kGenL2] += so;
    }
    if constexpr (DEG == 9) S[kGenL3] = F::acc(F::acc(S[kGenL3], Q, PG_TB(kR3P, j)), Q, PG_TB(kR3M, j));
    // a difference within rounding noise of zero (2^12 u of the magnitude
    // of its five values) says nothing about the axis: its sign bit marks it
    // for region_epilogue, which then skips it
    const double dj = fabs((si - 2.0 * f0) - q * (so - 2.0 * f0));
    // (for the positive families the values are their own magnitudes)
    const double mj = F::kUnitBounded
                          ? (fabs(pin) + fabs(min_)) + q * (fabs(pout) + fabs(mout)) + (2.0 + 2.0 * q) * fabs(f0)
                          : fma(2.0 + 2.0 * q, fabs(f0), fma(q, fabs(so), fabs(si)));
    D[j] = fma(-kDiffNoise, mj, dj) > 0.0 ? dj : -dj;
  }

  // axis pairs j < k: Q_jk = pre[j] * prod_{j<m<k} T0_m * suf[k+1]
#pragma unroll
  for (int j = 0; j < N - 1; ++j) {
    T PM = pre[j];
#pragma unroll
    for (int k = j + 1; k < N; ++k) {
      if (k > j + 1) PM = F::mul(PM, PG_TB(kC0, k - 1));
      T Q = (k == N - 1) ? PM : F::mul(PM, suf[k + 1]);
      T a1p = F::mul(Q, PG_TB(kR1P, j)), a1m = F::mul(Q, PG_TB(kR1M, j));
      const T b1p = PG_TB(kR1P, k), b1m = PG_TB(kR1M, k);
      double s5 = S[kGenL1L1];
      s5 = F::acc(s5, a1p, b1p);
      s5 = F::acc(s5, a1p, b1m);
      s5 = F::acc(s5, a1m, b1p);
      s5 = F::acc(s5, a1m, b1m);
      S[kGenL1L1] = s5;
      if constexpr (DEG == 9) {
        T a2p = F::mul(Q, PG_TB(kR2P, j)), a2m = F::mul(Q, PG_TB(kR2M, j));
        const T b2p = PG_TB(kR2P, k), b2m = PG_TB(kR2M, k);
        double s6 = S[kGenL1L2];
        s6 = F::acc(s6, a1p, b2p);
        s6 = F::acc(s6, a1p, b2m);
        s6 = F::acc(s6, a1m, b2p);
        s6 = F::acc(s6, a1m, b2m);
        s6 = F::acc(s6, a2p, b1p);
        s6 = F::acc(s6, a2p, b1m);
        s6 = F::acc(s6, a2m, b1p);
        s6 = F::acc(s6, a2m, b1m);
        S[kGenL1L2] = s6;
      }
    }
  }

  // axis triples j < k < l at l1: Q = pre[j] * mid(j,k) * mid(k,l) * suf[l+1]
  if (N >= 3 && DEG == 9) {
#pragma unroll
    for (int j = 0; j < N - 2; ++j) {
      T PM1 = pre[j];
#pragma unroll
      for (int k = j + 1; k < N - 1; ++k) {
        if (k > j + 1) PM1 = F::mul(PM1, PG_TB(kC0, k - 1));
        T aj[2] = {F::mul(PM1, PG_TB(kR1P, j)), F::mul(PM1, PG_TB(kR1M, j))};
        T ajk[4] = {F::mul(aj[0], PG_TB(kR1P, k)), F::mul(aj[0], PG_TB(kR1M, k)),
                    F::mul(aj[1], PG_TB(kR1P, k)), F::mul(aj[1], PG_TB(kR1M, k))};
        T MID = pre[0];  // identity placeholder until the first middle factor
        bool mid_id = true;
#pragma unroll
        for (int l = k + 1; l < N; ++l) {
          if (l > k + 1) {
            MID = mid_id ? PG_TB(kC0, l - 1) : F::mul(MID, PG_TB(kC0, l - 1));
            mid_id = false;
          }
          T C;
          bool c_id;
          if (l == N - 1) {
            C = MID;
            c_id = mid_id;
          } else {
            C = mid_id ? suf[l + 1] : F::mul(MID, suf[l + 1]);
            c_id = false;
          }
          // the remaining factor of each point, C t_l(+-), is shared by the
          // four sign pairs on (j, k)
          const T tp = c_id ? PG_TB(kR1P, l) : F::mul(C, PG_TB(kR1P, l));
          const T tm = c_id ? PG_TB(kR1M, l) : F::mul(C, PG_TB(kR1M, l));
#pragma unroll
          for (int s4 = 0; s4 < 4; ++s4) S[kGenL1L1L1] = F::acc(F::acc(S[kGenL1L1L1], ajk[s4], tp), ajk[s4], tm);
        }
      }
    }
  }

  // every axis at l0 (2^N sign vertices): split the axes into halves
  {
    constexpr int H1 = N / 2;
    constexpr int H2 = N - H1;
    T Bv[1 << H2];
    Bv[0] = PG_TB(kR0P, H1);
    Bv[1] = PG_TB(kR0M, H1);
#pragma unroll
    for (int t = 1; t < H2; ++t) {
      const T fp = PG_TB(kR0P, H1 + t), fm = PG_TB(kR0M, H1 + t);
#pragma unroll
      for (int s2 = (1 << t) - 1; s2 >= 0; --s2) {
        Bv[2 * s2 + 1] = F::mul(Bv[s2], fm);
        Bv[2 * s2] = F::mul(Bv[s2], fp);
      }
    }
    // the first half's sign products by the same doubling, the family's base
    // folded into its first axis
    T Av[1 << H1];
    Av[0] = F::mul(base, PG_TB(kR0P, 0));
    Av[1] = F::mul(base, PG_TB(kR0M, 0));
#pragma unroll
    for (int t = 1; t < H1; ++t) {
      const T fp = PG_TB(kR0P, t), fm = PG_TB(kR0M, t);
#pragma unroll
      for (int s1 = (1 << t) - 1; s1 >= 0; --s1) {
        Av[2 * s1 + 1] = F::mul(Av[s1], fm);
        Av[2 * s1] = F::mul(Av[s1], fp);
      }
    }
    double acc = 0.0;
#pragma unroll
    for (int s1 = 0; s1 < (1 << H1); ++s1)
#pragma unroll
      for (int s2 = 0; s2 < (1 << H2); ++s2) acc = F::acc(acc, Av[s1], Bv[s2]);
    S[kGenL0All] = acc;
  }
#undef PG_TB
}

// Rule, null rules, error and split axis of one region from its sums.
// UNIT: the integrand is signed with |f| <= 1, so the magnitude of an orbit
// sum is bounded by the orbit size; otherwise f > 0 and it is |S_g|.
// DEG 7: one null rule, w7 - w5, whose value is the error |R7 - R5|.
template <int N, bool UNIT, int DEG = 9>
__device__ __forceinline__ void region_epilogue(const EvalRule& R, const double (&S)[kNumGen], const double (&D)[N],
                                                double vol, const double (&width)[N], double& V, double& E, int& K,
                                                double* nk_out) {
  constexpr int NK = DEG == 9 ? 4 : 1;  // null rules in use
  double b = 0.0, u[4] = {0.0, 0.0, 0.0, 0.0}, msum = 0.0, vmag = 0.0;
#pragma unroll
  for (int g = 0; g < kNumGen; ++g) {
    if (DEG == 7 && !(g == kGenCentre || g == kGenL2 || g == kGenLp || g == kGenL1L1 || g == kGenL0All)) continue;
    b = fma(R.w[g][0], S[g], b);
#pragma unroll
    for (int k = 0; k < NK; ++k) u[k] = fma(R.w[g][1 + k], S[g], u[k]);
    if (!UNIT) {
      msum += fabs(S[g]);
      vmag = fma(fabs(R.w[g][0]), fabs(S[g]), vmag);
    }
  }
  V = vol * b;
  // null values at the rounding level of their own sums count as zero: the
  // floor is noise * vol * sum_g |u_kg| M_g; max_g |u_kg| * sum_g M_g bounds
  // it from above, so the exact floor is formed only when the bound does not
  // already clear N_k
  double nk[4] = {0.0, 0.0, 0.0, 0.0}, nu[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
  for (int k = 0; k < NK; ++k) {
    nk[k] = vol * fabs(u[k]);
    const double bound = UNIT ? R.floor_unit[k] : R.umax[k] * msum;
    double floor_k = 0.0;
    const bool need = nk[k] <= R.noise * (vol * bound);
    if (need || nk_out) {
      double sc = 0.0;
#pragma unroll
      for (int g = 0; g < kNumGen; ++g) sc = fma(fabs(R.w[g][1 + k]), UNIT ? R.cnt[g] : fabs(S[g]), sc);
      floor_k = R.noise * (vol * sc);
    }
    nu[k] = (need && nk[k] <= floor_k) ? 0.0 : nk[k];
    if (nk_out) {
      nk_out[k] = nk[k];
      nk_out[4 + k] = floor_k;
    }
  }
  if (nk_out)
#pragma unroll
    for (int k = NK; k < 4; ++k) nk_out[k] = nk_out[4 + k] = 0.0;
  E = DEG == 9 ? null_error(nu[0], nu[1], nu[2], nu[3]) : nu[0];
  // no error below the rounding level of V itself
  const double vround = kVRound * (vol * (UNIT ? R.vround_unit : vmag));
  if (E < vround) E = vround;
  // split axis: the largest fourth difference above its noise floor (floored
  // ones carry a negative sign), near-ties to the lowest axis; with every
  // difference at the floor, the widest axis
  double dmax = 0.0;
#pragma unroll
  for (int j = 0; j < N; ++j) dmax = fmax(dmax, D[j]);
  int k = 0;
  if (dmax > 0.0) {
    const double thr = (1.0 - 1e-10) * dmax;
    k = N - 1;
#pragma unroll
    for (int j = N - 1; j >= 0; --j)
      if (D[j] >= thr) k = j;
  } else {
#pragma unroll
    for (int j = 1; j < N; ++j)
      if (width[j] > width[k]) k = j;
  }
  K = k;
}

// ------------------------------------------------- cooperative evaluation
// Table entry (code, axis j) of the box [lo, lo + 2^-lv): the same
// expression as axis_entries (cache when the level is cached, else the
// factor), so both give the same bits.
template <class F>
__device__ __forceinline__ typename F::T entry_value(const EvalRule& R, const IntegrandParams& prm,
                                                     const typename F::T* __restrict__ cache, int cache_levels,
                                                     double lo, int lv, int j, int code) {
  if (cache != nullptr && lv <= cache_levels)
    return cache[((size_t)j * kCacheSlots + ((1 << lv) - 1) + dyadic_index(lo, lv)) * kCodes + code];
  const double h = 0.5 * pow2_neg(lv);
  return F::factor(F::axis(prm, j), point_x(prm, j, lo + h, h, code_offset(R, code)));
}

// One warp per sibling pair, 16 lanes per region: the lanes build the
// region's factor table together, take its rule points from the packed code
// list (each point the product of its n table entries), reduce the nine
// generator sums by butterfly, and compute one fourth difference each; then
// every lane runs the same epilogue as the thread-per-pair form and lane 0
// applies the two-level estimate and writes the pair.  Used while few pairs
// exist: a thread-per-pair pass over them would run a handful of warps
// through long dependent FP64 chains (about 64 cycles each) and a large
// instruction stream.  The per-thread partial sums it leaves (lane 0 of each
// warp) feed the block reduction of the loop kernel.
template <class F, int N, int THREADS, int DEG>
__device__ __forceinline__ void coop_pairs(const EvalRule& R, const LoopArgs& A, const IntegrandParams& prm,
                                           const double* __restrict__ lower, const uint8_t* __restrict__ level,
                                           int64_t cap, int64_t npairs, int it, int relerr, double tau_rel,
                                           typename F::T* smem_warp, NSum& sv, NSum& se, NSum& svol, double& emin,
                                           double& emax, long long& nrel, int& nonfinite) {
  typedef typename F::T T;
  const int lane = threadIdx.x & 31, half = lane >> 4, hl = lane & 15;
  const int64_t warp0 = ((int64_t)blockIdx.x * THREADS + threadIdx.x) >> 5;
  const int64_t nwarps = (int64_t)gridDim.x * (THREADS / 32);
  T* tab = smem_warp + half * (kCodes * N);  // [code][axis] of this half's region
  const T base = F::base(prm);
  const T* __restrict__ fcache = static_cast<const T*>(A.fcache);
  const uint64_t* __restrict__ codes = A.codes;
  for (int64_t p = warp0; p < npairs; p += nwarps) {
    const int64_t i = 2 * p + half;
    double lo_mine = 0.0;
    int lv_mine = 0;
    if (hl < N) {
      lo_mine = lower[(size_t)hl * cap + i];
      lv_mine = level[(size_t)hl * cap + i];
    }
    double lo[N];
    int lv[N], lvsum = 0;
#pragma unroll
    for (int j = 0; j < N; ++j) {
      lo[j] = __shfl_sync(0xffffffffu, lo_mine, half * 16 + j);
      lv[j] = __shfl_sync(0xffffffffu, lv_mine, half * 16 + j);
      lvsum += lv[j];
    }
    for (int e = hl; e < kCodes * N; e += 16) {
      const int code = e / N, j = e - code * N;
      double loj = lo[0];
      int lvj = lv[0];
#pragma unroll
      for (int m = 1; m < N; ++m)
        if (j == m) {
          loj = lo[m];
          lvj = lv[m];
        }
      tab[code * N + j] = entry_value<F>(R, prm, fcache, A.fcache_levels, loj, lvj, j, code);
    }
    __syncwarp();

    // generator sums, lanes strided over each orbit's points
    double S[kNumGen];
#pragma unroll
    for (int g = 0; g < kNumGen; ++g) {
      S[g] = 0.0;
      if (DEG == 7 && !(g == kGenCentre || g == kGenL2 || g == kGenLp || g == kGenL1L1 || g == kGenL0All)) continue;
      double acc = 0.0;
      for (int q = A.gen_off[g] + hl; q < A.gen_off[g + 1]; q += 16) {
        const uint64_t w = codes[q];
        T f = base;
#pragma unroll
        for (int j = 0; j < N; ++j) f = F::mul(f, tab[(int)((w >> (4 * j)) & 15) * N + j]);
        acc += F::val(f);
      }
      S[g] = acc;
    }
#pragma unroll
    for (int off = 8; off > 0; off >>= 1)
#pragma unroll
      for (int g = 0; g < kNumGen; ++g) S[g] += __shfl_xor_sync(0xffffffffu, S[g], off);

    // fourth difference of axis hl (the same formula and noise floor as
    // rule_sums), gathered to every lane of the half
    double Dj;
    {
      const int jd = hl < N ? hl : 0;
      constexpr bool kOut = DEG == 9 && F::kOuterSplit;
      constexpr int kInP = kOut ? kR2P : kRpP, kInM = kOut ? kR2M : kRpM;
      constexpr int kOutP = kOut ? kR1P : kR2P, kOutM = kOut ? kR1M : kR2M;
      T c0 = base, ip = base, im = base, op = base, om = base;
#pragma unroll
      for (int m = 0; m < N; ++m) {
        const T t0 = tab[kC0 * N + m];
        c0 = F::mul(c0, t0);
        ip = F::mul(ip, m == jd ? tab[kInP * N + m] : t0);
        im = F::mul(im, m == jd ? tab[kInM * N + m] : t0);
        op = F::mul(op, m == jd ? tab[kOutP * N + m] : t0);
        om = F::mul(om, m == jd ? tab[kOutM * N + m] : t0);
      }
      const double q = split_q<F, DEG>(R);
      const double f0 = F::val(c0), vip = F::val(ip), vim = F::val(im), vop = F::val(op), vom = F::val(om);
      const double si = vip + vim, so = vop + vom;
      const double dj = fabs((si - 2.0 * f0) - q * (so - 2.0 * f0));
      const double mj = F::kUnitBounded
                            ? (fabs(vip) + fabs(vim)) + q * (fabs(vop) + fabs(vom)) + (2.0 + 2.0 * q) * fabs(f0)
                            : fma(2.0 + 2.0 * q, fabs(f0), fma(q, fabs(so), fabs(si)));
      Dj = fma(-kDiffNoise, mj, dj) > 0.0 ? dj : -dj;
    }
    double D[N], width[N];
#pragma unroll
    for (int j = 0; j < N; ++j) {
      D[j] = __shfl_sync(0xffffffffu, Dj, half * 16 + j);
      width[j] = pow2_neg(lv[j]) * prm.len[j];
    }
    double V, E;
    int K;
    region_epilogue<N, F::kUnitBounded, DEG>(R, S, D, pow2_neg(lvsum) * prm.vol, width, V, E, K, nullptr);
    const double VR = __shfl_sync(0xffffffffu, V, 16);
    double ER = __shfl_sync(0xffffffffu, E, 16);
    const int KR = __shfl_sync(0xffffffffu, K, 16);
    const int lvR = __shfl_sync(0xffffffffu, lvsum, 16);
    if (lane == 0) {
      const double VL = V;
      double EL = E;
      if (it > 1) two_level(VL, VR, A.pool.Vp[p], EL, ER);
      *reinterpret_cast<double2*>(A.pool.V + 2 * p) = make_double2(VL, VR);
      *reinterpret_cast<double2*>(A.pool.E + 2 * p) = make_double2(EL, ER);
      *reinterpret_cast<uchar2*>(A.pool.K + 2 * p) = make_uchar2((unsigned char)K, (unsigned char)KR);
      const bool aL = relerr_active(VL, EL, tau_rel, relerr), aR = relerr_active(VR, ER, tau_rel, relerr);
      *reinterpret_cast<uchar2*>(A.pool.act + 2 * p) = make_uchar2(aL, aR);
      nadd(sv, VL);
      nadd(sv, VR);
      nadd(se, EL);
      nadd(se, ER);
      nadd(svol, pow2_neg(lvsum));
      nadd(svol, pow2_neg(lvR));
      emin = fmin(emin, fmin(EL, ER));
      emax = fmax(emax, fmax(EL, ER));
      nrel += aL + aR;
      if (!isfinite(VL) || !isfinite(VR) || !isfinite(EL) || !isfinite(ER)) nonfinite = 1;
    }
    __syncwarp();  // the table is rewritten for the next pair
  }
}

// ------------------------------------------------------------- loop kernel
// One thread per sibling pair (2p, 2p+1) of the current pool buffer; DEG is
// the rule (9, or 7 for the Genz-Malik variant).
template <class F, int N, int THREADS, int DEG = 9>
__global__ void __launch_bounds__(THREADS, PAGANI_EVAL_MINB) k_evaluate_loop(const EvalRule R, const LoopArgs A) {
  typedef typename F::T T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* tab = reinterpret_cast<T*>(smem_raw) + threadIdx.x;

  Ctrl& c = *A.ctrl;
  const int64_t s = c.s;
  const int it = c.it;
  const int buf = (it - 1) & 1;
  const int64_t cap = A.pool.cap;
  const double* __restrict__ lower = A.pool.lower + (size_t)buf * N * cap;
  const uint8_t* __restrict__ level = A.pool.level + (size_t)buf * N * cap;
  const double tau_rel = c.tau_cls;  // Rel-Err-Classify tolerance of this iteration
  const int relerr = c.relerr_filter;
  const IntegrandParams prm = *A.prm;
  const T base = F::base(prm);
  const T* __restrict__ fcache = static_cast<const T*>(A.fcache);

  NSum sv = {0.0, 0.0}, se = {0.0, 0.0}, svol = {0.0, 0.0};
  double emin = __longlong_as_double(0x7ff0000000000000LL), emax = -emin;
  long long nrel = 0;
  int nonfinite = 0;

  const int64_t npairs = s >> 1;
  const int64_t nwarps = (int64_t)gridDim.x * (THREADS / 32);
  const bool coop = A.codes != nullptr && npairs <= kCoopPasses * nwarps;
  const bool per_region = !coop && s <= (int64_t)kRegionPasses * gridDim.x * THREADS;
  if (coop) {
    // (parameters read through global memory: the cooperative table build
    // indexes them with a runtime axis, which must not move the kernel's
    // register copy to local memory)
    coop_pairs<F, N, THREADS, DEG>(R, A, *A.prm, lower, level, cap, npairs, it, relerr, tau_rel,
                                   reinterpret_cast<T*>(smem_raw) + (threadIdx.x >> 5) * 32 * kCodes * N, sv, se,
                                   svol, emin, emax, nrel, nonfinite);
  } else if (per_region) {
    // one thread per region; a warp covers 32 consecutive regions (16
    // sibling pairs) and stays converged for the sibling exchange
    const int lane = threadIdx.x & 31;
    for (int64_t r0 = (int64_t)blockIdx.x * THREADS + (threadIdx.x - lane); r0 < s;
         r0 += (int64_t)gridDim.x * THREADS) {
      const int64_t i = r0 + lane;
      const bool live = i < s;  // s is even: siblings are live together
      double V = 0.0, E = 0.0;
      int K = 0, lvsum = 0;
      if (live) {
        double wd[N];
#pragma unroll
        for (int j = 0; j < N; ++j) {
          const double lo = lower[(size_t)j * cap + i];
          const int lv = level[(size_t)j * cap + i];
          wd[j] = pow2_neg(lv) * prm.len[j];
          lvsum += lv;
          axis_entries<F, N, THREADS>(tab, R, prm, fcache, A.fcache_levels, lo, lv, j);
        }
        double S[kNumGen], D[N];
        rule_sums<F, N, THREADS, DEG>(tab, base, split_q<F, DEG>(R), S, D);
        region_epilogue<N, F::kUnitBounded, DEG>(R, S, D, pow2_neg(lvsum) * prm.vol, wd, V, E, K, nullptr);
      }
      const double Vo = __shfl_xor_sync(0xffffffffu, V, 1);
      const double Eo = __shfl_xor_sync(0xffffffffu, E, 1);
      if (live) {
        // both siblings form the same two-level estimate; each keeps its own
        const bool left = (lane & 1) == 0;
        const double VL = left ? V : Vo, VR = left ? Vo : V;
        double EL = left ? E : Eo, ER = left ? Eo : E;
        if (it > 1) two_level(VL, VR, A.pool.Vp[i >> 1], EL, ER);
        const double Em = left ? EL : ER;
        A.pool.V[i] = V;
        A.pool.E[i] = Em;
        A.pool.K[i] = (unsigned char)K;
        const bool a = relerr_active(V, Em, tau_rel, relerr);
        A.pool.act[i] = a;
        nadd(sv, V);
        nadd(se, Em);
        nadd(svol, pow2_neg(lvsum));
        emin = fmin(emin, Em);
        emax = fmax(emax, Em);
        nrel += a;
        if (!isfinite(V) || !isfinite(Em)) nonfinite = 1;
      }
    }
  } else
  for (int64_t p = (int64_t)blockIdx.x * THREADS + threadIdx.x; p < npairs; p += (int64_t)gridDim.x * THREADS) {
    const int64_t iL = 2 * p;
    double loL[N], loR[N], wL[N], wR[N];
    int lvLj[N];
    int lvL = 0, lvR = 0, diff_axis = -1, diff_lv = 0;
    double diff_lo = 0.0;
#pragma unroll
    for (int j = 0; j < N; ++j) {
      const double2 lo2 = *reinterpret_cast<const double2*>(lower + (size_t)j * cap + iL);
      const uchar2 lv2 = *reinterpret_cast<const uchar2*>(level + (size_t)j * cap + iL);
      loL[j] = lo2.x;
      loR[j] = lo2.y;
      // widths on the integration bounds (they only break split-axis ties)
      wL[j] = pow2_neg(lv2.x) * prm.len[j];
      wR[j] = pow2_neg(lv2.y) * prm.len[j];
      lvLj[j] = lv2.x;
      lvL += lv2.x;
      lvR += lv2.y;
      if (lo2.x != lo2.y || lv2.x != lv2.y) {
        diff_axis = j;
        diff_lo = lo2.y;
        diff_lv = lv2.y;
      }
    }
    // factor table of the left region
#pragma unroll
    for (int j = 0; j < N; ++j)
      axis_entries<F, N, THREADS>(tab, R, prm, fcache, A.fcache_levels, loL[j], lvLj[j], j);
    double S[kNumGen], D[N];
    double VL, EL, VR, ER;
    int KL, KR;
    rule_sums<F, N, THREADS, DEG>(tab, base, split_q<F, DEG>(R), S, D);
    region_epilogue<N, F::kUnitBounded, DEG>(R, S, D, pow2_neg(lvL) * prm.vol, wL, VL, EL, KL, nullptr);
    // patch the one axis where the right sibling differs
    if (diff_axis >= 0)
      axis_entries<F, N, THREADS>(tab, R, prm, fcache, A.fcache_levels, diff_lo, diff_lv, diff_axis);
    rule_sums<F, N, THREADS, DEG>(tab, base, split_q<F, DEG>(R), S, D);
    region_epilogue<N, F::kUnitBounded, DEG>(R, S, D, pow2_neg(lvR) * prm.vol, wR, VR, ER, KR, nullptr);

    if (it > 1) two_level(VL, VR, A.pool.Vp[p], EL, ER);

    *reinterpret_cast<double2*>(A.pool.V + iL) = make_double2(VL, VR);
    *reinterpret_cast<double2*>(A.pool.E + iL) = make_double2(EL, ER);
    *reinterpret_cast<uchar2*>(A.pool.K + iL) = make_uchar2((unsigned char)KL, (unsigned char)KR);
    // Rel-Err-Classify, kept per region for the probe and count kernels
    const bool aL = relerr_active(VL, EL, tau_rel, relerr), aR = relerr_active(VR, ER, tau_rel, relerr);
    *reinterpret_cast<uchar2*>(A.pool.act + iL) = make_uchar2(aL, aR);

    nadd(sv, VL);
    nadd(sv, VR);
    nadd(se, EL);
    nadd(se, ER);
    nadd(svol, pow2_neg(lvL));
    nadd(svol, pow2_neg(lvR));
    emin = fmin(emin, fmin(EL, ER));
    emax = fmax(emax, fmax(EL, ER));
    nrel += aL + aR;
    if (!isfinite(VL) || !isfinite(VR) || !isfinite(EL) || !isfinite(ER)) nonfinite = 1;
  }

  // block reduction of the partials (fixed order: deterministic).  A block
  // without pairs holds the identity and skips it (a warp-wide FP64
  // instruction occupies its scheduler's FP64 unit about 64 cycles), and the
  // last block combines only the partials of blocks that had pairs, which
  // leaves every sum bit for bit unchanged
  // (cooperative: pair p on warp p mod nwarps, THREADS/32 warps a block;
  // per region: region i on thread i mod (grid threads))
  const int64_t units = per_region ? s : npairs;
  const int64_t per_block = coop ? THREADS / 32 : THREADS;
  const int64_t nparts_eval = (units + per_block - 1) / per_block < (int64_t)gridDim.x
                                  ? (units + per_block - 1) / per_block
                                  : (int64_t)gridDim.x;
  if ((int64_t)blockIdx.x < nparts_eval) {
    EvalPartial mine;
    mine.v = sv;
    mine.e = se;
    mine.vol = svol;
    mine.emin = emin;
    mine.emax = emax;
    mine.n_rel = nrel;
    mine.nonfinite = nonfinite;
    mine.pad = 0;
    // (the factor tables in shared memory are done with: the reduction
    // stages its partials there)
    const EvalPartial bp = eval_block_finish<THREADS>(mine, smem_raw);
    if (threadIdx.x == 0) A.eval_part[blockIdx.x] = bp;
  }
  if (!last_block_arrived(&c.ticket_eval)) return;
  EvalPartial acc = eval_identity();
  for (int64_t b = threadIdx.x; b < nparts_eval; b += THREADS) acc = eval_combine(acc, A.eval_part[b]);
  const EvalPartial tot = eval_block_finish<THREADS>(acc, smem_raw);
  if (threadIdx.x == 0) {
    int search = finalize_iteration_head(c, nval(tot.v), nval(tot.e), tot.n_rel, tot.emin, tot.emax,
                                         tot.nonfinite, A.trace, A.trace_cap, nval(tot.vol));
    set_cond(A.use_graph, A.h_probe, (unsigned)search);
    __threadfence();
  }
}

// ------------------------------------------------------- factor-cache fill
// Fills every cached level (0 .. fcache_levels) of the per-axis factor cache
// in one launch before the loop: n (2^(levels+1) - 1) 11 factors, one thread
// per (axis, interval, code), with the expression axis_entries uses.
template <class F, int N>
__global__ void __launch_bounds__(256) k_factor_cache(const EvalRule R, const LoopArgs A) {
  typedef typename F::T T;
  if (A.fcache == nullptr) return;
  T* cache = static_cast<T*>(A.fcache);
  const IntegrandParams prm = *A.prm;
  const long long slots = (2LL << A.fcache_levels) - 1;
  const long long total = (long long)N * slots * kCodes;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int code = (int)(idx % kCodes);
    const long long rest = idx / kCodes;
    const long long slot = rest % slots;
    const int j = (int)(rest / slots);
    const int L = 63 - __clzll(slot + 1);       // slot = 2^L - 1 + k
    const long long k = slot + 1 - (1LL << L);
    const double w = pow2_neg(L);
    const double h = 0.5 * w;
    const double lo = (double)k * w;
    cache[((size_t)j * kCacheSlots + slot) * kCodes + code] =
        F::factor(F::axis(prm, j), point_x(prm, j, lo + h, h, code_offset(R, code)));
  }
}

// --------------------------------------------------------- standalone kernel
// Evaluates a caller-given list of boxes (lower, width SoA, n x m) with the
// null-rule error (no two-level refinement); pairs (2i, 2i+1) share a thread.
template <class F, int N, int THREADS, bool DIAG, int DEG = 9>
__global__ void __launch_bounds__(THREADS) k_evaluate_standalone(const EvalRule R, const StandaloneArgs A) {
  typedef typename F::T T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* tab = reinterpret_cast<T*>(smem_raw) + threadIdx.x;
  const IntegrandParams prm = *A.prm;
  const T base = F::base(prm);
  const int64_t m = A.m;
  const int64_t npairs = (m + 1) >> 1;
  for (int64_t p = (int64_t)blockIdx.x * THREADS + threadIdx.x; p < npairs; p += (int64_t)gridDim.x * THREADS) {
#pragma unroll
    for (int side = 0; side < 2; ++side) {
      const int64_t i = 2 * p + side;
      if (i >= m) break;
      double lo[N], w[N], vol = 1.0;
#pragma unroll
      for (int j = 0; j < N; ++j) {
        lo[j] = A.lower[(size_t)j * m + i];
        w[j] = A.width[(size_t)j * m + i];
        vol *= w[j];
      }
      // the right box reuses the left box's entries on every axis it shares
#pragma unroll
      for (int j = 0; j < N; ++j) {
        bool same = false;
        if (side == 1) same = (lo[j] == A.lower[(size_t)j * m + i - 1]) && (w[j] == A.width[(size_t)j * m + i - 1]);
        if (!same) {
          const double h = 0.5 * w[j];
          build_axis<F, N, THREADS>(tab, R, prm, lo[j] + h, h, j);
        }
      }
      double S[kNumGen], D[N], V, E, nk[8];
      int K;
      rule_sums<F, N, THREADS, DEG>(tab, base, split_q<F, DEG>(R), S, D);
      region_epilogue<N, F::kUnitBounded, DEG>(R, S, D, vol, w, V, E, K, nk);
      A.V[i] = V;
      A.E[i] = E;
      A.K[i] = K;
      if (DIAG) {
#pragma unroll
        for (int t = 0; t < 8; ++t) A.diag[(size_t)t * m + i] = nk[t];
#pragma unroll
        for (int j = 0; j < N; ++j) A.diag[(size_t)(8 + j) * m + i] = fabs(D[j]);
      }
    }
  }
}

// ------------------------------------------------- batched factor cache
// The per-instance factor cache of one (family, n) group: levels 0 ..
// kBatchCacheLevels of every axis, with the instance's own parameters and
// the expression axis_entries uses, so cached and computed entries agree.
template <class F, int N>
__global__ void __launch_bounds__(256) k_factor_cache_batch(const EvalRule R, const BatchArgs A, const BatchGroup G) {
  typedef typename F::T T;
  if (G.fcache == nullptr) return;
  T* cache = static_cast<T*>(G.fcache);
  const long long per_inst = (long long)N * kBatchCacheSlots * kCodes;
  const long long total = (long long)G.count * per_inst;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int li = (int)(idx / per_inst);
    const long long r = idx - (long long)li * per_inst;
    const int code = (int)(r % kCodes);
    const long long rest = r / kCodes;
    const long long slot = rest % kBatchCacheSlots;
    const int j = (int)(rest / kBatchCacheSlots);
    const int L = 63 - __clzll(slot + 1);  // slot = 2^L - 1 + k
    const long long k = slot + 1 - (1LL << L);
    const double w = pow2_neg(L);
    const double h = 0.5 * w;
    const double lo = (double)k * w;
    const IntegrandParams& prm = A.prm[G.first + li];
    cache[idx] = F::factor(F::axis(prm, j), point_x(prm, j, lo + h, h, code_offset(R, code)));
  }
}

// ------------------------------------------------------ batched evaluate
// Evaluate for one (family, n) group of a batch: one thread per sibling pair
// over every instance's slot of the group's pool; each pair reads its
// instance's parameters and iteration.  Writes V (rule), E (null-rule error
// refined by the two-level estimate from the second iteration on) and K; the
// per-instance sums are taken by the batch reduce kernel.
template <class F, int N, int THREADS>
__global__ void __launch_bounds__(THREADS) k_evaluate_batch(const EvalRule R, const BatchArgs A,
                                                            const BatchGroup G) {
  typedef typename F::T T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* tab = reinterpret_cast<T*>(smem_raw) + threadIdx.x;
  const int64_t slots = (int64_t)G.count * G.slot_cap;
  // live pairs only: thread t's pair belongs to the instance whose prefix
  // range holds it (binary search over the group's instances)
  const long long* __restrict__ pre = A.pair_prefix;
  const long long first = pre[G.first];
  const long long npairs = pre[G.first + G.count] - first;
  for (long long t = (long long)blockIdx.x * THREADS + threadIdx.x; t < npairs; t += (long long)gridDim.x * THREADS) {
    const long long key = first + t;
    int lo_i = 0, hi_i = G.count - 1;  // last instance with pre[G.first + li] <= key
    while (lo_i < hi_i) {
      const int mid = (lo_i + hi_i + 1) >> 1;
      if (pre[G.first + mid] <= key) lo_i = mid;
      else hi_i = mid - 1;
    }
    const int li = lo_i;
    const Ctrl& c = A.inst[G.first + li].c;
    const int64_t p = (int64_t)li * (G.slot_cap >> 1) + (key - pre[G.first + li]);  // group pair index
    const int64_t iL = 2 * p;
    const int it = c.it;
    const int buf = (it - 1) & 1;
    const double* __restrict__ lower = G.lower + (size_t)buf * N * slots;
    const uint8_t* __restrict__ level = G.level + (size_t)buf * N * slots;
    const IntegrandParams& prm = A.prm[G.first + li];
    const T base = F::base(prm);
    const T* __restrict__ icache =
        G.fcache ? static_cast<const T*>(G.fcache) + (size_t)li * N * kBatchCacheSlots * kCodes : nullptr;
    double loL[N], wL[N], wR[N];
    int lvLj[N];
    int lvL = 0, lvR = 0, diff_axis = -1, diff_lv = 0;
    double diff_lo = 0.0;
#pragma unroll
    for (int j = 0; j < N; ++j) {
      const double2 lo2 = *reinterpret_cast<const double2*>(lower + (size_t)j * slots + iL);
      const uchar2 lv2 = *reinterpret_cast<const uchar2*>(level + (size_t)j * slots + iL);
      loL[j] = lo2.x;
      wL[j] = pow2_neg(lv2.x) * prm.len[j];
      wR[j] = pow2_neg(lv2.y) * prm.len[j];
      lvLj[j] = lv2.x;
      lvL += lv2.x;
      lvR += lv2.y;
      if (lo2.x != lo2.y || lv2.x != lv2.y) {
        diff_axis = j;
        diff_lo = lo2.y;
        diff_lv = lv2.y;
      }
    }
#pragma unroll
    for (int j = 0; j < N; ++j)
      axis_entries<F, N, THREADS, kBatchCacheSlots>(tab, R, prm, icache, kBatchCacheLevels, loL[j], lvLj[j], j);
    double S[kNumGen], D[N];
    double VL, EL, VR, ER;
    int KL, KR;
    rule_sums<F, N, THREADS>(tab, base, split_q<F, 9>(R), S, D);
    region_epilogue<N, F::kUnitBounded>(R, S, D, pow2_neg(lvL) * prm.vol, wL, VL, EL, KL, nullptr);
    if (diff_axis >= 0)
      axis_entries<F, N, THREADS, kBatchCacheSlots>(tab, R, prm, icache, kBatchCacheLevels, diff_lo, diff_lv,
                                                    diff_axis);
    rule_sums<F, N, THREADS>(tab, base, split_q<F, 9>(R), S, D);
    region_epilogue<N, F::kUnitBounded>(R, S, D, pow2_neg(lvR) * prm.vol, wR, VR, ER, KR, nullptr);
    if (it > 1) two_level(VL, VR, G.Vp[p], EL, ER);
    *reinterpret_cast<double2*>(G.V + iL) = make_double2(VL, VR);
    *reinterpret_cast<double2*>(G.E + iL) = make_double2(EL, ER);
    *reinterpret_cast<uchar2*>(G.K + iL) = make_uchar2((unsigned char)KL, (unsigned char)KR);
  }
}

// ---------------------------------------------------------------- launchers
template <class F, int N, int THREADS, int DEG = 9>
cudaError_t launch_loop(const EvalRule& R, const LoopArgs& A, int grid, int block, size_t smem, cudaStream_t st) {
  k_evaluate_loop<F, N, THREADS, DEG><<<grid, block, smem, st>>>(R, A);
  return cudaGetLastError();
}
template <class F, int N>
cudaError_t launch_fill(const EvalRule& R, const LoopArgs& A, int grid, int block, size_t smem, cudaStream_t st) {
  k_factor_cache<F, N><<<grid, block, smem, st>>>(R, A);
  return cudaGetLastError();
}
template <class F, int N, int THREADS, bool DIAG, int DEG = 9>
cudaError_t launch_standalone(const EvalRule& R, const StandaloneArgs& A, int grid, int block, size_t smem,
                              cudaStream_t st) {
  k_evaluate_standalone<F, N, THREADS, DIAG, DEG><<<grid, block, smem, st>>>(R, A);
  return cudaGetLastError();
}

template <class F, int N>
cudaError_t launch_batch_fill(const EvalRule& R, const BatchArgs& A, const BatchGroup& G, int grid, cudaStream_t st) {
  k_factor_cache_batch<F, N><<<grid, 256, 0, st>>>(R, A, G);
  return cudaGetLastError();
}
template <class F, int N, int THREADS>
cudaError_t launch_batch_eval(const EvalRule& R, const BatchArgs& A, const BatchGroup& G, int grid, cudaStream_t st) {
  k_evaluate_batch<F, N, THREADS><<<grid, THREADS, sizeof(typename F::T) * kCodes * N * THREADS, st>>>(R, A, G);
  return cudaGetLastError();
}

}  // namespace pg
