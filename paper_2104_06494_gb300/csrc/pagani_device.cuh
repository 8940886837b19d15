// Device helpers shared by the evaluate kernels and the region-management
// kernels: compensated sums, block reductions, and the per-iteration decisions
// of the PAGANI loop (Algorithm 2: termination test, Threshold-Classify
// trigger; Algorithm 3: one step of the threshold search).
#pragma once
#include <cstdint>
#include <cstring>

#include "pagani_internal.h"

namespace pg {

// Neumaier compensated summation.
__host__ __device__ __forceinline__ void nadd(NSum& a, double x) {
  double t = a.s + x;
  double big = fabs(a.s) >= fabs(x) ? a.s : x;
  double small = fabs(a.s) >= fabs(x) ? x : a.s;
  a.c += (big - t) + small;
  a.s = t;
}
__host__ __device__ __forceinline__ NSum ncomb(NSum a, const NSum& b) {
  nadd(a, b.s);
  a.c += b.c;
  return a;
}
__host__ __device__ __forceinline__ double nval(const NSum& a) { return a.s + a.c; }

__device__ __forceinline__ NSum shfl_down_nsum(NSum a, int off) {
  NSum b;
  b.s = __shfl_down_sync(0xffffffffu, a.s, off);
  b.c = __shfl_down_sync(0xffffffffu, a.c, off);
  return b;
}

// Width 2^-l as an exact double built from its exponent bits (integer ops only).
__device__ __forceinline__ double pow2_neg(int l) {
  return __longlong_as_double((long long)(1023 - l) << 52);
}

// Region error from the four null-rule values N1..N4 (degrees 7, 5, 3, 1),
// the reading of Sec. 3.2 used throughout.  On a resolved box the values fall
// off geometrically with the degree, by r per two degrees, and the rule's own
// error is about r N1:
//   r = max(N1/N2, N2/N3, N3/N4) with x/0 = inf (x > 0) or 0 (x = 0);
//   r >= 1 (no decay): 10 max(N1, N2, N3);
//   r < 1: 10 r max(N1, r N2)  (r N2 replaces a degree-7 value that cancelled
//   by accident).
// The caller passes N_k = 0 for values at the rounding level of their own
// sums and applies the rounding floor of V afterwards.
__device__ __forceinline__ double ratio_or(double x, double y) {
  return y > 0.0 ? x / y : (x > 0.0 ? __longlong_as_double(0x7ff0000000000000LL) : 0.0);
}
__device__ __forceinline__ double null_error(double n1, double n2, double n3, double n4) {
  const double r = fmax(fmax(ratio_or(n1, n2), ratio_or(n2, n3)), ratio_or(n3, n4));
  if (r >= 1.0) return 10.0 * fmax(fmax(n1, n2), n3);
  return 10.0 * r * fmax(n1, r * n2);
}

// Two-level error refinement of a sibling pair (Sec. 3.2), as read here: with
// delta = |V_L + V_R - V_parent| / 4 and S = E_L + E_R, each error becomes
// E (1 + 2 delta / S) + delta (E + delta when S = 0).
__device__ __forceinline__ void two_level(double VL, double VR, double Vpar, double& EL, double& ER) {
  double delta = fabs(VL + VR - Vpar) / 4.0;
  double S = EL + ER;
  if (S > 0.0) {
    double c = 1.0 + 2.0 * delta / S;
    EL = EL * c + delta;
    ER = ER * c + delta;
  } else {
    EL += delta;
    ER += delta;
  }
}

// Rel-Err-Classify (Sec. 3.5.1): active unless E <= tau |V|, with tau the
// loop's classification tolerance c.tau_cls.
__device__ __forceinline__ bool relerr_active(double V, double E, double tau, int enabled) {
  return enabled ? !(E <= tau * fabs(V)) : true;
}

// The next iteration's Rel-Err-Classify tolerance: the survivors' share of
// what the tolerance still allows, min(tau_rel, (tau_rel |v_tot| - e_f) /
// |sum of the survivors' V|).  The Lemma of Sec. 3.5.1 then keeps the error
// of regions finished by it within that allowance; before any threshold
// commit it is tau_rel itself for a same-sign integrand.  A share below
// tau_rel is rounded down to a power of two (its exponent bits kept, its
// mantissa cleared): once most of the tolerance is spent the allowance is a
// difference of nearly equal sums, whose rounding must not move the
// classification.
// The largest power of two not above x > 0 (its exponent bits kept, the
// mantissa cleared; a subnormal keeps its highest bit).
__host__ __device__ __forceinline__ double pow2_floor(double x) {
  unsigned long long bits;
  memcpy(&bits, &x, sizeof(bits));
  if ((bits >> 52) == 0) {
    while (bits & (bits - 1)) bits &= bits - 1;
  } else {
    bits &= 0xFFF0000000000000ULL;
  }
  double out;
  memcpy(&out, &bits, sizeof(out));
  return out;
}
// The smallest power of two not below x > 0.
__host__ __device__ __forceinline__ double pow2_ceil(double x) {
  const double f = pow2_floor(x);
  return f == x ? x : 2.0 * f;
}
__host__ __device__ __forceinline__ double survivor_tolerance(double tau_rel, double v_tot, double ef,
                                                              double v_surv) {
  const double allow = tau_rel * fabs(v_tot) - ef;
  if (!(allow < tau_rel * fabs(v_surv))) return tau_rel;
  if (!(allow > 0.0)) return 0.0;
  return pow2_floor(allow / fabs(v_surv));
}

// Final classification of a region after the optional threshold search.
__device__ __forceinline__ bool final_active(double V, double E, const Ctrl& c) {
  bool a = relerr_active(V, E, c.tau_cls, c.relerr_filter);
  if (c.search_ok) a = a && !(E < c.t);
  return a;
}

// Last-block election: every block calls this after publishing its partial;
// exactly one (the last to arrive) gets true and may read all partials.
__device__ __forceinline__ bool last_block_arrived(unsigned int* ticket, unsigned int nblocks) {
  __shared__ bool is_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned int prev = atomicAdd(ticket, 1u);
    is_last = (prev == nblocks - 1);
  }
  __syncthreads();
  if (is_last) {
    __threadfence();
    if (threadIdx.x == 0) *ticket = 0u;  // reset for the next launch
  }
  return is_last;
}
__device__ __forceinline__ bool last_block_arrived(unsigned int* ticket) {
  return last_block_arrived(ticket, gridDim.x);
}

// ---------------------------------------------------------------------------
// Combining per-block partials in the last block.  A one-lane FP64 instruction
// occupies the FP64 pipe like a full warp's, so the partials are combined by
// every thread of the block (a strided pass, then warp shuffles and a fixed
// warp order: the result is deterministic for a fixed grid).
__device__ __forceinline__ EvalPartial eval_identity() {
  EvalPartial p;
  p.v.s = p.v.c = p.e.s = p.e.c = p.vol.s = p.vol.c = 0.0;
  p.emin = __longlong_as_double(0x7ff0000000000000LL);
  p.emax = -p.emin;
  p.n_rel = 0;
  p.nonfinite = 0;
  p.pad = 0;
  return p;
}
__device__ __forceinline__ EvalPartial eval_combine(EvalPartial a, const EvalPartial& b) {
  a.v = ncomb(a.v, b.v);
  a.e = ncomb(a.e, b.e);
  a.vol = ncomb(a.vol, b.vol);
  a.emin = fmin(a.emin, b.emin);
  a.emax = fmax(a.emax, b.emax);
  a.n_rel += b.n_rel;
  a.nonfinite |= b.nonfinite;
  return a;
}
__device__ __forceinline__ EvalPartial eval_shfl(const EvalPartial& a, int off) {
  EvalPartial b;
  b.v = shfl_down_nsum(a.v, off);
  b.e = shfl_down_nsum(a.e, off);
  b.vol = shfl_down_nsum(a.vol, off);
  b.emin = __shfl_down_sync(0xffffffffu, a.emin, off);
  b.emax = __shfl_down_sync(0xffffffffu, a.emax, off);
  b.n_rel = __shfl_down_sync(0xffffffffu, a.n_rel, off);
  b.nonfinite = __shfl_down_sync(0xffffffffu, a.nonfinite, off);
  b.pad = 0;
  return b;
}
template <int THREADS>
__device__ __forceinline__ EvalPartial eval_block_combine(EvalPartial acc, EvalPartial* sh) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc = eval_combine(acc, eval_shfl(acc, off));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0)
    for (int w = 1; w < THREADS / 32; ++w) acc = eval_combine(acc, sh[w]);
  return acc;  // valid on thread 0
}

// K compensated sums reduced over the block through shared memory: a
// warp-wide FP64 instruction occupies its scheduler's FP64 unit about 64
// cycles on this GPU, so the reduction keeps the number of them small
// instead of running every warp through a shuffle tree.  The K x THREADS partials are staged in sh; K*32
// threads fold chunks of THREADS/32 consecutive partials in index order, and
// warp k reduces sum k's 32 chunk results by shuffles.  Fixed order:
// deterministic.  sh holds K * THREADS + K sums; the results are valid on
// thread 0 (in a).  With fewer warps than sums, a warp takes several.
template <int THREADS, int K>
__device__ __forceinline__ void nsum_block_reduce_staged(NSum (&a)[K], NSum* sh) {
  constexpr int C = THREADS / 32;  // partials per chunk: 32 chunks per sum
  constexpr int NW = THREADS / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
#pragma unroll
  for (int k = 0; k < K; ++k) sh[k * THREADS + threadIdx.x] = a[k];
  __syncthreads();
  for (int k = warp; k < K; k += NW) {
    const NSum* src = sh + k * THREADS + lane * C;
    NSum r = src[0];
#pragma unroll
    for (int t = 1; t < C; ++t) r = ncomb(r, src[t]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) r = ncomb(r, shfl_down_nsum(r, off));
    if (lane == 0) sh[K * THREADS + k] = r;
  }
  __syncthreads();
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < K; ++k) a[k] = sh[K * THREADS + k];
}

// An EvalPartial reduced over the block: the three compensated sums staged
// as above; emin / emax as the bit patterns of non-negative doubles (their
// integer order is the numeric one; the -inf of an empty partial is a
// negative integer), so no FP64 instruction is spent on them.  smem holds
// 3 * THREADS + 3 sums plus 4 * THREADS/32 64-bit words.  Valid on thread 0.
template <int THREADS>
__device__ __forceinline__ EvalPartial eval_block_finish(EvalPartial p, void* smem) {
  constexpr int NW = THREADS / 32;
  NSum* shn = static_cast<NSum*>(smem);
  long long* shl = reinterpret_cast<long long*>(shn + 3 * THREADS + 3);
  NSum a3[3] = {p.v, p.e, p.vol};
  long long imin = __double_as_longlong(p.emin), imax = __double_as_longlong(p.emax), nrel = p.n_rel;
  int nf = p.nonfinite;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const long long a = __shfl_down_sync(0xffffffffu, imin, off), b = __shfl_down_sync(0xffffffffu, imax, off);
    imin = a < imin ? a : imin;
    imax = b > imax ? b : imax;
    nrel += __shfl_down_sync(0xffffffffu, nrel, off);
    nf |= __shfl_down_sync(0xffffffffu, nf, off);
  }
  nsum_block_reduce_staged<THREADS, 3>(a3, shn);  // begins and ends with a barrier
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    shl[warp] = imin;
    shl[NW + warp] = imax;
    shl[2 * NW + warp] = nrel;
    shl[3 * NW + warp] = nf;
  }
  __syncthreads();
  EvalPartial out = p;
  if (threadIdx.x == 0) {
    for (int w = 1; w < NW; ++w) {
      imin = shl[w] < imin ? shl[w] : imin;
      imax = shl[NW + w] > imax ? shl[NW + w] : imax;
      nrel += shl[2 * NW + w];
      nf |= (int)shl[3 * NW + w];
    }
    out.v = a3[0];
    out.e = a3[1];
    out.vol = a3[2];
    out.emin = __longlong_as_double(imin);
    out.emax = __longlong_as_double(imax);
    out.n_rel = nrel;
    out.nonfinite = nf;
    out.pad = 0;
  }
  return out;
}

// Exclusive scan of one 64-bit count per thread across the block (thread
// order), by warp shuffles; *total receives the sum (all threads).
template <int THREADS>
__device__ __forceinline__ long long block_exclusive_scan(long long x, long long* sh, long long* total) {
  constexpr int NW = THREADS / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  long long inc = x;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const long long y = __shfl_up_sync(0xffffffffu, inc, off);
    if (lane >= off) inc += y;
  }
  __syncthreads();
  if (lane == 31) sh[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    long long t = lane < NW ? sh[lane] : 0;
#pragma unroll
    for (int off = 1; off < NW; off <<= 1) {
      const long long y = __shfl_up_sync(0xffffffffu, t, off);
      if (lane >= off) t += y;
    }
    if (lane < NW) sh[NW + lane] = t;  // inclusive warp offsets
  }
  __syncthreads();
  *total = sh[2 * NW - 1];
  return inc - x + (warp > 0 ? sh[NW + warp - 1] : 0);
}

__device__ __forceinline__ void set_cond(int use_graph, cudaGraphConditionalHandle h, unsigned int v) {
  if (use_graph) cudaGraphSetConditional(h, v);
}

// Decisions after Evaluate, Two-Level-Error, Rel-Err-Classify and the sums
// (Algorithm 2, from the termination test to the Threshold-Classify trigger).
// Runs on one thread.  Returns 1 if a threshold search starts.
__device__ inline int finalize_iteration_head(Ctrl& c, double v, double e, long long n_rel, double emin,
                                              double emax, int nonfinite, TraceRec* trace, int trace_cap,
                                              double vol) {
  c.active_volume = vol;
  c.v = v;
  c.e = e;
  c.n_rel = n_rel;
  c.emin = emin;
  c.emax = emax;
  c.n_regions_total += c.s;
  c.search = 0;
  c.search_ok = 0;
  c.trigger = 0;
  c.probes = 0;
  c.passes = 0;
  c.dir_changes = 0;
  c.t = 0.0;
  if (nonfinite || !isfinite(v) || !isfinite(e)) {
    c.status = -6;
    c.done = 1;
    c.estimate = v + c.vf;
    c.errorest = e + c.ef;
    return 0;
  }
  TraceRec tr = {};
  tr.it = c.it;
  tr.s = c.s;
  tr.v = v;
  tr.e = e;
  tr.vf = c.vf;
  tr.ef = c.ef;
  tr.n_relerr_active = n_rel;
  bool conv = (e + c.ef) / fabs(v + c.vf) <= c.tau_rel || e + c.ef <= c.tau_abs;
  if (conv || c.it >= c.it_max) {
    c.status = conv ? 0 : 1;
    c.done = 1;
    c.estimate = v + c.vf;
    c.errorest = e + c.ef;
    if (c.trace_on && c.it - 1 < trace_cap) trace[c.it - 1] = tr;
    return 0;
  }
  double v_tot = v + c.vf;
  int trig = 0;
  // c.heuristic_filter is the mask of enabled triggers (bit 0 digits, bit 1 memory)
  if ((c.heuristic_filter & 1) && c.it >= 2 && fabs(v_tot - c.v_tot_prev) <= c.tau_rel * fabs(v_tot)) trig |= 1;
  if ((c.heuristic_filter & 2) && 2 * n_rel > c.max_regions) trig |= 2;
  c.v_tot_prev = v_tot;
  c.trigger = trig;
  tr.trigger = trig;
  if (c.trace_on && c.it - 1 < trace_cap) trace[c.it - 1] = tr;
  c.search_cont = 0;
  if (!trig) return 0;
  // Algorithm 3 set-up: P_max = .25, t = e_it / s_it, and the error budget
  // e_b = tau_rel |v_tot| - e_f: what finished regions may still add before
  // the tolerance is out of reach (Sec. 3.5.3), rounded down to a power of
  // two (near the end a difference of nearly equal sums, its low bits the
  // rounding of e_f)
  c.Pmax = 0.25;
  c.e_b = fabs(v_tot) * c.tau_rel - c.ef;
  if (c.e_b > 0.0) c.e_b = pow2_floor(c.e_b);
  // the start (the mean error) and the range [min E, max E] rounded to
  // powers of two, the mean and the minimum down, the maximum up: errors
  // carry the rounding of the null-rule and two-level differences they come
  // from, and rounded inputs make every threshold of the search reproducible
  c.t = e / (double)c.s;
  if (c.t > 0.0) c.t = pow2_floor(c.t);
  if (c.emin > 0.0) c.emin = pow2_floor(c.emin);
  if (c.emax > 0.0) c.emax = pow2_ceil(c.emax);
  c.last_dir = 0;
  if (!(c.e_b > 0.0)) return 0;
  c.search = 1;
  c.search_cont = 1;
  return 1;
}

// The fields of the control block that the steps of the search read and
// write, held in registers while one thread takes several steps in a row.
struct SearchState {
  int64_t s;
  int32_t probes, total_probes, search_ok, last_dir, dir_changes;
  double t, Pmax, e_b, emin, emax;
  __device__ explicit SearchState(const Ctrl& c)
      : s(c.s), probes(c.probes), total_probes(c.total_probes), search_ok(c.search_ok), last_dir(c.last_dir),
        dir_changes(c.dir_changes), t(c.t), Pmax(c.Pmax), e_b(c.e_b), emin(c.emin), emax(c.emax) {}
  // the fields a step changes, back into the control block
  __device__ void store(Ctrl& c) const {
    c.probes = probes;
    c.total_probes = total_probes;
    c.search_ok = search_ok;
    c.last_dir = last_dir;
    c.dir_changes = dir_changes;
    c.t = t;
    c.Pmax = Pmax;
  }
};

// The threshold after t in the search of Algorithm 3: too few regions
// finished (dir > 0) moves it halfway to max E, too much error (dir < 0)
// halfway to min E.  The probe kernel builds its tree of coming thresholds
// with this same function, so they are the bits threshold_step arrives at.
__host__ __device__ __forceinline__ double search_next(double t, int dir, double emin, double emax) {
  return dir > 0 ? t + (emax - t) / 2.0 : t - (t - emin) / 2.0;
}

// One step of Algorithm 3 after a probe with threshold c.t counted
// n_active candidate actives; e_abar is the error of the candidate finished
// regions (summed directly, not as e_it - sum A.E).  Returns 1 if another
// probe is needed.  S is the control block or a register copy of its search
// fields (SearchState) with the same names.
template <class S>
__device__ inline int threshold_step(S& c, long long n_active, double e_abar) {
  c.probes += 1;
  c.total_probes += 1;
  long long s_abar = c.s - n_active;
  int dir;
  if (2 * s_abar > c.s) {                          // memory requirement, s_abar > 0.5 s
    if (e_abar <= c.Pmax * c.e_b) {               // accuracy requirement
      c.search_ok = 1;
      return 0;
    }
    dir = -1;
  } else {
    dir = +1;
  }
  if (c.last_dir != 0 && dir != c.last_dir) {
    c.dir_changes += 1;
    c.Pmax = fmin(c.Pmax + 0.10, 0.95);
  }
  c.last_dir = dir;
  if (c.dir_changes >= 10 || c.probes >= 64) return 0;  // unsuccessful filtering
  c.t = search_next(c.t, dir, c.emin, c.emax);
  return 1;
}

}  // namespace pg
