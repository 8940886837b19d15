// Host side of the GB300 PAGANI engine: the region-management kernels of
// Algorithm 2 (Uniform-Split, the Threshold-Classify probes, the finished
// accumulation with the survivor count and its scan, and Filter + parent
// update + Split fused into one compaction kernel), the workspace, the
// device-resident loop as one CUDA graph with conditional WHILE nodes, and
// the C ABI declared in include/pagani.h.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/pagani.h"
#include "pagani_device.cuh"
#include "pagani_internal.h"

namespace pg {

static thread_local std::string g_err;

static int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

// ------------------------------------------------------ block-level helpers
template <int THREADS>
__device__ __forceinline__ long long block_sum_ll(long long x, long long* sh) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(0xffffffffu, x, off);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[warp] = x;
  __syncthreads();
  long long t = 0;
  if (threadIdx.x == 0)
    for (int w = 0; w < THREADS / 32; ++w) t += sh[w];
  return t;  // valid on thread 0
}

// Exclusive scan of one flag per thread across the block, in thread order.
// Returns this thread's rank among the set flags; *total = number set.
template <int THREADS>
__device__ __forceinline__ int block_rank(bool flag, int* sh, int* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned ballot = __ballot_sync(0xffffffffu, flag);
  const int within = __popc(ballot & ((1u << lane) - 1u));
  __syncthreads();
  if (lane == 0) sh[warp] = __popc(ballot);
  __syncthreads();
  int before = 0, tot = 0;
#pragma unroll
  for (int w = 0; w < THREADS / 32; ++w) {
    const int v = sh[w];
    before += (w < warp) ? v : 0;
    tot += v;
  }
  *total = tot;
  return before + within;
}

// ------------------------------------------------------------ Uniform-Split
// Region i of the d^n grid; axis n-1 varies fastest (Sec. 3.1).
__global__ void k_uniform_split(Pool P, int d, int log2d, int64_t s0) {
  const int n = P.n;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < s0; i += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = i;
    for (int j = n - 1; j >= 0; --j) {
      const int digit = (int)(r & (d - 1));  // d is a power of two
      r >>= log2d;
      P.lower[(size_t)j * P.cap + i] = (double)digit / (double)d;
      P.level[(size_t)j * P.cap + i] = (uint8_t)log2d;
    }
  }
}

// ------------------------------------------------- Threshold-Classify probe
// Bit pattern of a non-negative double (errors and thresholds); with the
// sign bit cleared, these order like the numbers, so E >= t is an integer
// comparison and costs no FP64 issue slot.
__device__ __forceinline__ unsigned long long ebits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFULL;
}

// E as an unsigned 128-bit fixed-point multiple of the error budget:
// floor(E 2^kProbeFrac / e_b) for E < e_b (below 2^kProbeFrac), and exactly
// 2^kProbeFrac (the budget itself) for E >= e_b.  e_b = 2^B is a power of
// two, so this is a shift of E's significand; integer operations only.
// e_bits: the bit pattern of e_b.
__device__ __forceinline__ void probe_fixed(unsigned long long eb, unsigned long long e_bits, int B,
                                            unsigned long long& lo, unsigned long long& hi) {
  if (eb >= e_bits) {
    lo = 0ull;
    hi = 1ull << (kProbeFrac - 64);
    return;
  }
  int ex = (int)(eb >> 52);
  unsigned long long m = eb & ((1ull << 52) - 1);
  if (ex) m |= 1ull << 52;
  else ex = 1;
  // E = m 2^(ex - 1075); E 2^(kProbeFrac - B) = m 2^sh, below 2^kProbeFrac.
  // PTX shifts clamp the shift amount to the register width (a shift by 64
  // or more gives 0), so every case (sh >= 64, 0 < sh < 64, sh = 0, sh < 0,
  // down to sh <= -64) is the same straight-line code: the warp does not
  // diverge on the errors' exponents.
  const int sh = ex - 1075 + kProbeFrac - B;
  const unsigned left = sh > 0 ? (unsigned)sh : 0u, right = sh < 0 ? (unsigned)(-sh) : 0u;
  const unsigned up = left < 64u ? 64u - left : 64u, down = left >= 64u ? left - 64u : 64u;
  unsigned long long l, r, h1, h2;
  asm("shl.b64 %0, %1, %2;" : "=l"(l) : "l"(m), "r"(left));
  asm("shr.b64 %0, %1, %2;" : "=l"(r) : "l"(l), "r"(right));
  asm("shr.b64 %0, %1, %2;" : "=l"(h1) : "l"(m), "r"(up));
  asm("shl.b64 %0, %1, %2;" : "=l"(h2) : "l"(m), "r"(down));
  lo = r;
  hi = h1 | h2;
}

// The probe's thresholds: node k of the coming steps of the search from t.
// Nodes 0..kProbeTree-1 form a binary tree in heap order (children 2k+1 one
// step down, 2k+2 one step up); the kProbeExt nodes after them continue the
// all-down path past the tree's depth, the last kProbeExt the all-up path.
constexpr int kProbeExt = kProbeRay - kProbeDepth + 1;
__device__ __forceinline__ double probe_node(int k, double t, double emin, double emax) {
  if (k < kProbeTree) {
    // directions from the root: the bits of k + 1 below its leading one
    const int x = k + 1;
    for (int b = 30 - __clz(x); b >= 0; --b) t = search_next(t, ((x >> b) & 1) ? 1 : -1, emin, emax);
    return t;
  }
  const bool up = k >= kProbeTree + kProbeExt;
  const int steps = kProbeDepth + (k - kProbeTree - (up ? kProbeExt : 0));
  for (int i = 0; i < steps; ++i) t = search_next(t, up ? 1 : -1, emin, emax);
  return t;
}
// The node after k when the search moves in direction d, or -1 when that
// threshold is not among the pass's nodes.
__device__ __forceinline__ int probe_next(int k, int d) {
  constexpr int kLeft = kProbeTree / 2, kRight = kProbeTree - 1;  // the all-down and all-up leaves
  if (k < kLeft) return d < 0 ? 2 * k + 1 : 2 * k + 2;
  if (k < kProbeTree) return k == kLeft && d < 0 ? kProbeTree : (k == kRight && d > 0 ? kProbeTree + kProbeExt : -1);
  if (k < kProbeTree + kProbeExt) return d < 0 && k + 1 < kProbeTree + kProbeExt ? k + 1 : -1;
  return d > 0 && k + 1 < kProbeNodes ? k + 1 : -1;
}

// Threshold-Classify (Algorithm 3): one probe pass takes the search from the
// current threshold t through as many of its steps as the pass's thresholds
// cover: any kProbeDepth steps, and up to kProbeRay steps that keep one
// direction.  The thresholds are computed here with search_next, the
// function threshold_step moves by, so they are the bits the search arrives
// at.  Every block places each region's error among the sorted thresholds
// and adds it to its bucket (rel-err actives) or to the finished bin; the
// bins hold exact integer sums (probe_fixed) and counts, combined over the
// grid by integer atomics.  The last block then takes the steps of
// Algorithm 3 with those totals: at a threshold, the candidate actives are
// the rel-err actives of the buckets above it and e_abar is the error of the
// buckets below it plus the rel-err finished.  The pass ends when the search
// ends or moves to a threshold it does not cover; a following pass starts
// from the threshold it left in c.t.
template <int THREADS>
__global__ void __launch_bounds__(THREADS) k_probe(const LoopArgs A) {
  Ctrl& c = *A.ctrl;
  constexpr int NW = THREADS / 32;
  static_assert(kProbeNodes <= 31 && THREADS >= 32, "one warp computes the nodes; 32 sorted entries");
  __shared__ unsigned long long nodeb[kProbeNodes];    // node k's threshold bits
  __shared__ int node_at[kProbeNodes];                 // the first sorted threshold equal to node k's
  __shared__ unsigned long long thr[32];               // sorted thresholds, padded with all ones
  __shared__ ulonglong2 hist[kProbeBins * THREADS];    // per thread: (lo, hi | count << 44) per bin
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t s = c.s;
  const int64_t np = (s + 1) / 2;
  // only the first nact blocks have region pairs: the others leave at once,
  // and the last of the nact to arrive takes the search's steps
  const int64_t need = (np + THREADS - 1) / THREADS;
  const unsigned nact = need < 1 ? 1u : (need < (int64_t)gridDim.x ? (unsigned)need : gridDim.x);
  if (blockIdx.x >= nact) return;
  if (threadIdx.x < kProbeNodes) nodeb[threadIdx.x] = ebits(probe_node(threadIdx.x, c.t, c.emin, c.emax));
#pragma unroll
  for (int b = 0; b < kProbeBins; ++b) hist[b * THREADS + threadIdx.x] = make_ulonglong2(0ull, 0ull);
  __syncthreads();
  if (threadIdx.x < kProbeNodes) {
    // rank among the nodes (equal values by node index)
    const unsigned long long x = nodeb[threadIdx.x];
    int below = 0, r = 0;
    for (int j = 0; j < kProbeNodes; ++j) {
      below += nodeb[j] < x;
      r += nodeb[j] < x || (nodeb[j] == x && j < (int)threadIdx.x);
    }
    thr[r] = x;
    node_at[threadIdx.x] = below;
  } else if (threadIdx.x < 32) {
    thr[threadIdx.x] = ~0ull;
  }
  __syncthreads();
  const unsigned long long e_bits = ebits(c.e_b);
  int B;  // e_b = 2^B
  if (e_bits >> 52) B = (int)(e_bits >> 52) - 1023;
  else B = -1074 + 63 - __clzll((long long)e_bits);
  const uint8_t* __restrict__ act = A.pool.act;
  const double* __restrict__ E = A.pool.E;
  ulonglong2* mine = hist + threadIdx.x;
  auto add = [&](unsigned long long eb, int a) {
    // number of thresholds at or below E (branch-free search of 32 entries)
    int k = thr[15] <= eb ? 16 : 0;
    k += thr[k + 7] <= eb ? 8 : 0;
    k += thr[k + 3] <= eb ? 4 : 0;
    k += thr[k + 1] <= eb ? 2 : 0;
    k += thr[k] <= eb ? 1 : 0;
    const int bin = a ? k : kProbeBuckets;
    unsigned long long lo, hi;
    probe_fixed(eb, e_bits, B, lo, hi);
    ulonglong2 h = mine[bin * THREADS];
    h.x += lo;
    h.y += hi + (h.x < lo ? 1ull : 0ull) + (1ull << 44);
    mine[bin * THREADS] = h;
  };
  // regions in pairs (one 16-byte load of two errors, one 2-byte load of two
  // classification bytes), U pairs per thread in flight; E and act hold
  // cap >= s + 1 entries for odd s (cap is a multiple of 4096), and the
  // entry past s is masked
  constexpr int U = 4;
  const int64_t stride = (int64_t)gridDim.x * THREADS;
  const double2* __restrict__ E2 = reinterpret_cast<const double2*>(E);
  const uint16_t* __restrict__ act2 = reinterpret_cast<const uint16_t*>(act);
  for (int64_t p0 = (int64_t)blockIdx.x * THREADS + threadIdx.x; p0 < np; p0 += U * stride) {
    double2 e2[U];
    unsigned a2[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t p = p0 + u * stride;
      e2[u] = p < np ? E2[p] : make_double2(0.0, 0.0);
      a2[u] = p < np ? (unsigned)act2[p] : 0u;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t p = p0 + u * stride;
      if (p >= np) break;
      add(ebits(e2[u].x), (int)(a2[u] & 0xff));
      if (2 * p + 1 < s) add(ebits(e2[u].y), (int)(a2[u] >> 8));
    }
  }
  __syncthreads();
  // per bin: the block's sum and count, then one set of atomics
  for (int b = warp; b < kProbeBins; b += NW) {
    unsigned long long lo = 0ull, hi = 0ull, cnt = 0ull;
#pragma unroll
    for (int t = lane; t < THREADS; t += 32) {
      const ulonglong2 h = hist[b * THREADS + t];
      lo += h.x;
      hi += (h.y & ((1ull << 44) - 1)) + (lo < h.x ? 1ull : 0ull);
      cnt += h.y >> 44;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const unsigned long long lo2 = __shfl_down_sync(0xffffffffu, lo, off);
      const unsigned long long hi2 = __shfl_down_sync(0xffffffffu, hi, off);
      const unsigned long long c2 = __shfl_down_sync(0xffffffffu, cnt, off);
      lo += lo2;
      hi += hi2 + (lo < lo2 ? 1ull : 0ull);
      cnt += c2;
    }
    if (lane == 0 && cnt != 0ull) {
      constexpr unsigned long long M44 = (1ull << 44) - 1;
      ProbeAcc& g = A.probe_acc[b];
      atomicAdd(&g.limb[0], lo & M44);
      atomicAdd(&g.limb[1], (lo >> 44) | ((hi & ((1ull << 24) - 1)) << 20));
      atomicAdd(&g.limb[2], hi >> 24);
      atomicAdd(&g.cnt, cnt);
    }
  }
  if (!last_block_arrived(&c.ticket_probe, nact)) return;
  // the grid's bins, then at every threshold (in parallel) the candidate
  // actives and e_abar; thread 0 then takes the steps
  __shared__ unsigned long long blo[kProbeBins], bhi[kProbeBins], bcnt[kProbeBins];
  __shared__ long long n_at[kProbeNodes];
  __shared__ double e_at[kProbeNodes];
  if (threadIdx.x < kProbeBins) {
    ProbeAcc& g = A.probe_acc[threadIdx.x];
    const unsigned long long l0 = __ldcg(&g.limb[0]), l1 = __ldcg(&g.limb[1]), l2 = __ldcg(&g.limb[2]);
    bcnt[threadIdx.x] = __ldcg(&g.cnt);
    g.limb[0] = g.limb[1] = g.limb[2] = g.cnt = 0ull;  // zero for the next pass
    const unsigned long long a = l1 << 44;
    const unsigned long long lo = l0 + a;
    blo[threadIdx.x] = lo;
    bhi[threadIdx.x] = (l1 >> 20) + (l2 << 24) + (lo < a ? 1ull : 0ull);
  }
  __syncthreads();
  if (threadIdx.x < kProbeNodes) {
    // at the sorted threshold j: the candidate actives are the rel-err
    // actives of buckets j+1.., e_abar the error of buckets 0..j plus the
    // rel-err finished
    const int j = threadIdx.x;
    long long na = 0;
    for (int b = j + 1; b < kProbeBuckets; ++b) na += (long long)bcnt[b];
    unsigned long long lo = blo[kProbeBuckets], hi = bhi[kProbeBuckets];
    for (int b = 0; b <= j; ++b) {
      lo += blo[b];
      hi += bhi[b] + (lo < blo[b] ? 1ull : 0ull);
    }
    n_at[j] = na;
    e_at[j] = scalbn(fma(__ull2double_rn(hi), 0x1p64, __ull2double_rn(lo)), B - kProbeFrac);
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  c.passes += 1;
  c.total_passes += 1;
  // the steps run on a register copy of the search fields: one read of the
  // control block before them and one write after, not a round trip to
  // memory per field and step
  SearchState st(c);
  int k = 0, cont = 1;
  for (;;) {
    const int j = node_at[k];
    cont = threshold_step(st, n_at[j], e_at[j]);
    if (!cont) break;
    k = probe_next(k, st.last_dir);
    if (k < 0) break;  // not among this pass's thresholds: the next pass starts at c.t
    if (ebits(st.t) != nodeb[k]) {  // the step must land on the node's threshold, bit for bit
      c.watchdog = 3;
      st.search_ok = 0;
      cont = 0;
      break;
    }
  }
  st.store(c);
  c.search_cont = cont;
  set_cond(A.use_graph, A.h_probe, (unsigned)cont);
  __threadfence();
}

// ------------------------------------------------------------ survivor count
// The final classification of every region (Evaluate's Rel-Err-Classify
// byte and, after a successful threshold search, E >= t) and the survivors
// of every 256-region warp slice of a tile.  The last block takes the
// decisions that follow Threshold-Classify in Algorithm 2 that need only the
// survivor count (the memory check, Sec. 3.5.2).  The finished regions' sums
// (v_f, e_f of Algorithm 2) are formed by the split kernel, which reads
// every region's classification byte anyway.
//
// Built for bandwidth: the kernel does no floating-point arithmetic.  Each
// block owns a contiguous range of tiles; a thread takes ITEMS contiguous
// regions of a tile (one 8-byte load of their classification bytes), the
// bytes of kCountAhead tiles are requested before the first is used, and
// every warp stores its own slice count.  Without a search it reads one
// byte per region; after one, also E of each rel-err active region.  Each
// block scans its own tiles' counts (offsets within the block) and publishes
// its survivor total; the last block scans only the block totals.
constexpr int kCountAhead = 8;
constexpr int kCountEFrac = 96;

// add x = m 2^sh (m < 2^53) to the 128-bit (lo, hi); sh < 128
__device__ __forceinline__ void add128_shifted(unsigned long long& lo, unsigned long long& hi, unsigned long long m,
                                               int sh) {
  unsigned long long xl, xh;
  if (sh >= 64) {
    xl = 0ull;
    xh = m << (sh - 64);
  } else if (sh > 0) {
    xl = m << sh;
    xh = m >> (64 - sh);
  } else if (sh > -64) {
    xl = m >> (-sh);
    xh = 0ull;
  } else {
    return;
  }
  lo += xl;
  hi += xh + (lo < xl ? 1ull : 0ull);
}

// E (0 <= E <= 2^X) as a multiple of 2^(X - kCountEFrac), truncated, added to (lo, hi)
__device__ __forceinline__ void add_e_fixed(unsigned long long& lo, unsigned long long& hi, double e, int X) {
  const unsigned long long b = ebits(e);
  int ex = (int)(b >> 52);
  unsigned long long m = b & ((1ull << 52) - 1);
  if (ex) m |= 1ull << 52;
  else ex = 1;
  add128_shifted(lo, hi, m, ex - 1075 + kCountEFrac - X);
}

// 128-bit sums over a warp (valid on lane 0)
__device__ __forceinline__ void warp_sum128(unsigned long long& lo, unsigned long long& hi) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const unsigned long long l2 = __shfl_down_sync(0xffffffffu, lo, off);
    const unsigned long long h2 = __shfl_down_sync(0xffffffffu, hi, off);
    lo += l2;
    hi += h2 + (lo < l2 ? 1ull : 0ull);
  }
}

// (lo, hi) added to three 44-bit-limb accumulators by independent atomics
__device__ __forceinline__ void atomic_add_limbs(unsigned long long* limb, unsigned long long lo, unsigned long long hi) {
  constexpr unsigned long long M44 = (1ull << 44) - 1;
  atomicAdd(&limb[0], lo & M44);
  atomicAdd(&limb[1], (lo >> 44) | ((hi & ((1ull << 24) - 1)) << 20));
  atomicAdd(&limb[2], hi >> 24);
}
// the 128-bit value of three limb accumulators (read, then zeroed)
__device__ __forceinline__ void take_limbs(unsigned long long* limb, unsigned long long& lo, unsigned long long& hi) {
  const unsigned long long l0 = __ldcg(&limb[0]), l1 = __ldcg(&limb[1]), l2 = __ldcg(&limb[2]);
  limb[0] = limb[1] = limb[2] = 0ull;
  const unsigned long long a = l1 << 44;
  lo = l0 + a;
  hi = (l1 >> 20) + (l2 << 24) + (lo < a ? 1ull : 0ull);
}

// a 128-bit integer times 2^e as a double (nearly exact: two roundings)
__device__ __forceinline__ double fixed_to_double(unsigned long long lo, unsigned long long hi, int e) {
  return scalbn(fma(__ull2double_rn(hi), 0x1p64, __ull2double_rn(lo)), e);
}

// the exponent X of max E rounded up to a power of two, 2^X (E's fixed-point scale)
__device__ __forceinline__ int emax_scale(double emax) {
  const unsigned long long mb = ebits(emax);
  return (mb >> 52) ? (int)(mb >> 52) - 1023 + ((mb & ((1ull << 52) - 1)) ? 1 : 0) : -1022;
}

template <int THREADS, int ITEMS>
__global__ void __launch_bounds__(THREADS) k_count(const LoopArgs A) {
  static_assert(ITEMS == 8 && THREADS / 32 == kTileWarps, "one 8-byte load per thread, one slice per warp");
  Ctrl& c = *A.ctrl;
  if (c.done) {
    if (blockIdx.x == 0 && threadIdx.x == 0) set_cond(A.use_graph, A.h_main, 0u);
    return;
  }
  constexpr int TILE = THREADS * ITEMS;
  const int64_t s = c.s;
  const double* __restrict__ E = A.pool.E;
  uint8_t* __restrict__ act = A.pool.act;
  const int64_t ntiles = (s + TILE - 1) / TILE;
  const int64_t tpb = (ntiles + gridDim.x - 1) / gridDim.x;  // tiles per block
  // blocks past the last tile leave at once; the nact others take tickets
  const int64_t need = tpb > 0 ? (ntiles + tpb - 1) / tpb : 0;
  const unsigned nact = need < 1 ? 1u : (unsigned)need;
  if (blockIdx.x >= nact) return;
  const int64_t t_beg = (int64_t)blockIdx.x * tpb;
  const int64_t t_end = t_beg + tpb < ntiles ? t_beg + tpb : ntiles;
  const bool searched = c.search_ok != 0;
  const unsigned long long tb = ebits(c.t);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __shared__ long long shl[2 * (THREADS / 32)];
  // the classification bytes of kCountAhead tiles; the act array holds
  // cap >= s entries, cap a multiple of 4096: the 8-byte loads stay inside
  // it, and bytes past s are masked below
  auto load_bytes = [&](int64_t t0, unsigned long long (&b)[kCountAhead]) {
#pragma unroll
    for (int u = 0; u < kCountAhead; ++u) {
      const int64_t tile = t0 + u;
      const int64_t i0 = tile * TILE + (int64_t)threadIdx.x * ITEMS;
      b[u] = tile < t_end && i0 < s ? *reinterpret_cast<const unsigned long long*>(act + i0) : 0ull;
    }
  };
  unsigned long long bytes[kCountAhead], ahead[kCountAhead];
  if (t_beg < t_end) load_bytes(t_beg, bytes);
  for (int64_t t0 = t_beg; t0 < t_end; t0 += kCountAhead) {
    // the next group's bytes are in flight while this group is counted
    if (t0 + kCountAhead < t_end) load_bytes(t0 + kCountAhead, ahead);
#pragma unroll
    for (int u = 0; u < kCountAhead; ++u) {
      const int64_t tile = t0 + u;
      if (tile >= t_end) break;
      const int64_t i0 = tile * TILE + (int64_t)threadIdx.x * ITEMS;
      const int valid = i0 < s ? (s - i0 < ITEMS ? (int)(s - i0) : ITEMS) : 0;
      int cnt = 0;
      if (searched) {
        // rel-err actives the threshold finishes: E < t; their byte is
        // cleared for the split
        double ee[ITEMS];
        bool a0[ITEMS];
#pragma unroll
        for (int r = 0; r < ITEMS; ++r) {
          a0[r] = r < valid && ((bytes[u] >> (8 * r)) & 0xff) != 0;
          ee[r] = a0[r] ? E[i0 + r] : 0.0;
        }
#pragma unroll
        for (int r = 0; r < ITEMS; ++r) {
          const bool keep = a0[r] && ebits(ee[r]) >= tb;
          cnt += keep;
          if (a0[r] && !keep) act[i0 + r] = 0;
        }
      } else {
#pragma unroll
        for (int r = 0; r < ITEMS; ++r) cnt += r < valid && ((bytes[u] >> (8 * r)) & 0xff) != 0;
      }
      const int wc = __reduce_add_sync(0xffffffffu, cnt);
      if (lane == 0) A.pool.tile_count[tile * kTileWarps + warp] = wc;
    }
#pragma unroll
    for (int u = 0; u < kCountAhead; ++u) bytes[u] = ahead[u];
  }
  __syncthreads();  // the block's slice counts are written
  // survivors before each of the block's tiles, within the block: each
  // thread a contiguous chunk of tiles, the chunk sums scanned by shuffles
  auto tile_total = [&](int64_t t) {
    const int4* w = reinterpret_cast<const int4*>(A.pool.tile_count + t * kTileWarps);
    const int4 a = w[0], b = w[1];
    return (long long)a.x + a.y + a.z + a.w + b.x + b.y + b.z + b.w;
  };
  const int64_t nt = t_end > t_beg ? t_end - t_beg : 0;
  const int64_t per = (nt + THREADS - 1) / THREADS;
  const int64_t q0 = t_beg + (int64_t)threadIdx.x * per, q1 = q0 + per < t_end ? q0 + per : t_end;
  long long acc = 0;
  for (int64_t t = q0; t < q1; ++t) acc += tile_total(t);
  long long blk_surv = 0;
  long long run = block_exclusive_scan<THREADS>(acc, shl, &blk_surv);
  for (int64_t t = q0; t < q1; ++t) {
    const long long x = tile_total(t);
    A.pool.tile_offset[t] = run;
    run += x;
  }
  if (threadIdx.x == 0) A.count_part[blockIdx.x].n_surv = nt > 0 ? blk_surv : 0;
  if (!last_block_arrived(&c.ticket_count, nact)) return;

  // survivors before each block (the split adds them to the block's tile
  // offsets)
  const int G = (int)nact;
  const int per_b = (G + THREADS - 1) / THREADS;
  const int b0 = threadIdx.x * per_b, b1 = b0 + per_b < G ? b0 + per_b : G;
  long long bacc = 0;
  for (int b = b0; b < b1; ++b) bacc += __ldcg(&A.count_part[b].n_surv);
  long long n_surv = 0;
  long long brun = block_exclusive_scan<THREADS>(bacc, shl, &n_surv);
  for (int b = b0; b < b1; ++b) {
    const long long x = __ldcg(&A.count_part[b].n_surv);
    A.count_part[b].surv_before = brun;
    brun += x;
  }
  if (threadIdx.x != 0) return;
  c.count_tpb = tpb;
  c.n_surv = n_surv;
  const bool tr_ok = c.trace_on && c.it - 1 < A.trace_cap;
  TraceRec* tr = tr_ok ? &A.trace[c.it - 1] : nullptr;
  if (tr) {
    tr->trigger = c.trigger;
    tr->n_survivors = n_surv;
    if (c.trigger) {
      tr->probes = c.probes;
      tr->probe_passes = c.passes;
      tr->search_ok = c.search_ok;
      tr->threshold = c.t;
      tr->direction_changes = (double)c.dir_changes;
    }
  }
  if (2 * n_surv > c.max_regions) {  // memory exhausted (Sec. 3.5.2)
    c.status = 2;
    c.done = 1;
    c.estimate = c.v + c.vf;
    c.errorest = c.e + c.ef;
  }
  // independent bound on the device loop: never more than it_max + 1 passes
  c.loop_guard += 1;
  if (!c.done && c.loop_guard > c.it_max) {
    c.watchdog = 2;
    c.done = 1;
  }
  set_cond(A.use_graph, A.h_main, c.done ? 0u : 1u);
  __threadfence();
}

// ------------------------- Filter + parent update + Split + finished sums
// Survivor i with rank r (in region order) writes V_p[r] = V_i and its two
// halves along K_i to slots 2r (lower half) and 2r+1 (upper half) of the
// other pool buffer.  Every finished region adds its V, its E and its volume
// to the iteration's finished sums (v - sum V.A and e - sum E.A of Algorithm
// 2, formed directly over the finished regions): V as a plain per-thread sum
// of its items entering a Neumaier block sum, E and the volume exactly as
// integers (E as a fixed-point multiple of max E rounded up to a power of
// two, 2^-kCountEFrac of it; a volume 2^-L as 2^(127 - L), exact for
// L <= 127).  The last block then updates v_f, e_f and the survivors'
// classification share tau_cls, or, when no region survived, ends the loop
// (the it_max status: v + v_f and e + e_f cannot change any more).
template <int THREADS, int ITEMS>
__global__ void __launch_bounds__(THREADS, 2) k_split(const LoopArgs A) {
  Ctrl& c = *A.ctrl;
  const bool logl = c.keep_leaves && A.leaves.lower != nullptr;
  if (c.done) {
    // the integration ended in this iteration: every box of it is a leaf
    if (logl) {
      const int64_t s = c.s, base = c.leaf_count, cap = A.pool.cap, lcap = A.leaves.cap;
      const int n = A.pool.n, src = (c.it - 1) & 1;
      if (base + s > lcap && blockIdx.x == 0 && threadIdx.x == 0) atomicExch(&c.leaf_overflow, 1);
      for (int64_t i = (int64_t)blockIdx.x * THREADS + threadIdx.x; i < s; i += (int64_t)gridDim.x * THREADS) {
        if (base + i >= lcap) break;
        for (int j = 0; j < n; ++j) {
          A.leaves.lower[(size_t)j * lcap + base + i] = A.pool.lower[((size_t)src * n + j) * cap + i];
          A.leaves.level[(size_t)j * lcap + base + i] = A.pool.level[((size_t)src * n + j) * cap + i];
        }
      }
    }
    return;
  }
  constexpr int TILE = THREADS * ITEMS;
  const int64_t s = c.s;
  const int n = A.pool.n;
  const int64_t cap = A.pool.cap;
  const int src = (c.it - 1) & 1, dst = src ^ 1;
  const double* __restrict__ lo_s = A.pool.lower + (size_t)src * n * cap;
  const uint8_t* __restrict__ lv_s = A.pool.level + (size_t)src * n * cap;
  double* __restrict__ lo_d = A.pool.lower + (size_t)dst * n * cap;
  uint8_t* __restrict__ lv_d = A.pool.level + (size_t)dst * n * cap;
  const int64_t ntiles = (s + TILE - 1) / TILE;
  // blocks without a tile leave at once; the nact others take tickets
  const unsigned nact = ntiles < 1 ? 1u : (ntiles < (int64_t)gridDim.x ? (unsigned)ntiles : gridDim.x);
  if (blockIdx.x >= nact) return;
  const int X = emax_scale(c.emax);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int NW = THREADS / 32;
  __shared__ int shr[NW];
  __shared__ NSum shn[THREADS + 1];
  __shared__ unsigned long long shu[4 * NW];
  int bad = 0;
  NSum accv = {0.0, 0.0};
  unsigned long long elo = 0ull, ehi = 0ull, vlo = 0ull, vhi = 0ull;  // finished E and volume
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    // survivors before the tile: within its block of the count kernel, plus
    // before that block
    const long long tile_base = A.pool.tile_offset[tile] + A.count_part[tile / c.count_tpb].surv_before;
    // phase 1: every item's classification (stored by the count kernel) and
    // rank; phase 2: the loads and copies, whose loads then overlap across
    // items instead of following one barrier each
    bool actv[ITEMS], valid[ITEMS];
    long long qv[ITEMS];
#pragma unroll
    for (int r = 0; r < ITEMS; ++r) {
      const int64_t i = tile * TILE + (int64_t)r * THREADS + threadIdx.x;
      valid[r] = i < s;
      actv[r] = valid[r] && A.pool.act[i] != 0;  // classified by the count kernel
    }
    long long base = tile_base;
#pragma unroll
    for (int r = 0; r < ITEMS; ++r) {
      int total;
      const int rank = block_rank<THREADS>(actv[r], shr, &total);
      qv[r] = base + rank;
      base += total;
    }
    if (logl) {
#pragma unroll
      for (int r = 0; r < ITEMS; ++r) {
        const int64_t i = tile * TILE + (int64_t)r * THREADS + threadIdx.x;
        if (!actv[r] && valid[r]) {
          // finished box: its rank among the finished ones is i - (survivors before i)
          const int64_t pos = c.leaf_count + i - qv[r];
          if (pos < A.leaves.cap) {
            for (int j = 0; j < n; ++j) {
              A.leaves.lower[(size_t)j * A.leaves.cap + pos] = lo_s[(size_t)j * cap + i];
              A.leaves.level[(size_t)j * A.leaves.cap + pos] = lv_s[(size_t)j * cap + i];
            }
          } else {
            bad |= 2;
          }
        }
      }
    }
    // every item's loads are issued before any store (per axis), so a
    // thread waits on one L2 round trip per axis instead of one per item
    // and axis: V of every region, K of the survivors, E of the finished
    int kv[ITEMS], lsum[ITEMS];
    double vv[ITEMS], ev[ITEMS];
#pragma unroll
    for (int r = 0; r < ITEMS; ++r) {
      const int64_t i = tile * TILE + (int64_t)r * THREADS + threadIdx.x;
      kv[r] = actv[r] ? A.pool.K[i] : -1;
      vv[r] = valid[r] ? A.pool.V[i] : 0.0;
      ev[r] = valid[r] && !actv[r] ? A.pool.E[i] : 0.0;
      lsum[r] = 0;
    }
#pragma unroll
    for (int r = 0; r < ITEMS; ++r)
      if (actv[r]) A.pool.Vp[qv[r]] = vv[r];
    // the finished items' V and E (their volume follows from the levels)
    double tv = 0.0;
#pragma unroll
    for (int r = 0; r < ITEMS; ++r)
      if (valid[r] && !actv[r]) {
        tv += vv[r];
        add_e_fixed(elo, ehi, ev[r], X);
      }
    nadd(accv, tv);
    for (int j = 0; j < n; ++j) {
      double lo[ITEMS];
      int lv[ITEMS];
#pragma unroll
      for (int r = 0; r < ITEMS; ++r) {
        const int64_t i = tile * TILE + (int64_t)r * THREADS + threadIdx.x;
        lo[r] = actv[r] ? lo_s[(size_t)j * cap + i] : 0.0;
        lv[r] = valid[r] ? lv_s[(size_t)j * cap + i] : 0;  // the finished need it for their volume
      }
#pragma unroll
      for (int r = 0; r < ITEMS; ++r) {
        lsum[r] += lv[r];
        if (!actv[r]) continue;
        const int64_t q = qv[r];
        double2 out = make_double2(lo[r], lo[r]);
        uchar2 ol = make_uchar2((unsigned char)lv[r], (unsigned char)lv[r]);
        if (j == kv[r]) {
          if (lv[r] >= 62) bad = 1;
          out.y = lo[r] + pow2_neg(lv[r] + 1);
          ol = make_uchar2((unsigned char)(lv[r] + 1), (unsigned char)(lv[r] + 1));
        }
        *reinterpret_cast<double2*>(lo_d + (size_t)j * cap + 2 * q) = out;
        *reinterpret_cast<uchar2*>(lv_d + (size_t)j * cap + 2 * q) = ol;
      }
    }
#pragma unroll
    for (int r = 0; r < ITEMS; ++r)
      if (valid[r] && !actv[r]) add128_shifted(vlo, vhi, 1ull, 127 - lsum[r]);
  }
  if (bad & 1) atomicExch(&c.watchdog, 1);
  if (bad & 2) atomicExch(&c.leaf_overflow, 1);
  // the block's finished V (compensated), and E and volume (integers, added
  // to the grid totals in the control block by atomics)
  NSum v1[1] = {accv};
  nsum_block_reduce_staged<THREADS, 1>(v1, shn);
  warp_sum128(elo, ehi);
  warp_sum128(vlo, vhi);
  if (lane == 0) {
    shu[warp] = elo;
    shu[NW + warp] = ehi;
    shu[2 * NW + warp] = vlo;
    shu[3 * NW + warp] = vhi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < NW; ++w) {
      elo += shu[w];
      ehi += shu[NW + w] + (elo < shu[w] ? 1ull : 0ull);
      vlo += shu[2 * NW + w];
      vhi += shu[3 * NW + w] + (vlo < shu[2 * NW + w] ? 1ull : 0ull);
    }
    if (elo | ehi) atomic_add_limbs(c.fin_e_fixed, elo, ehi);
    if (vlo | vhi) atomic_add_limbs(c.fin_vol_fixed, vlo, vhi);
    A.count_part[blockIdx.x].va = v1[0];
  }
  if (!last_block_arrived(&c.ticket_split, nact)) return;
  NSum p1[1] = {{0.0, 0.0}};
  for (int b = threadIdx.x; b < (int)nact; b += THREADS)
    p1[0] = ncomb(p1[0], NSum{__ldcg(&A.count_part[b].va.s), __ldcg(&A.count_part[b].va.c)});
  nsum_block_reduce_staged<THREADS, 1>(p1, shn);
  if (threadIdx.x != 0) return;
  const NSum tva = p1[0];
  unsigned long long el, eh, vl, vh;
  take_limbs(c.fin_e_fixed, el, eh);  // (and zero them for the next iteration)
  take_limbs(c.fin_vol_fixed, vl, vh);
  const double tea = fixed_to_double(el, eh, X - kCountEFrac);
  const NSum tfv = {fixed_to_double(0ull, vh, -127), fixed_to_double(vl, 0ull, -127)};
  const double vf_new = c.vf + nval(tva);
  const double ef_new = c.ef + tea;
  const bool tr_ok = c.trace_on && c.it - 1 < A.trace_cap;
  if (tr_ok) {
    A.trace[c.it - 1].vf = vf_new;
    A.trace[c.it - 1].ef = ef_new;
  }
  if (c.n_surv == 0) {
    // nothing left to refine: v + v_f and e + e_f cannot change any more,
    // so the loop ends as it would at it_max (every box of the iteration was
    // finished, and logged as a leaf above)
    c.status = 1;
    c.done = 1;
    c.estimate = c.v + c.vf;
    c.errorest = c.e + c.ef;
    set_cond(A.use_graph, A.h_main, 0u);
  } else {
    c.tau_cls = survivor_tolerance(c.tau_rel, c.v + c.vf, ef_new, c.v - nval(tva));
    c.vf = vf_new;
    c.ef = ef_new;
    c.fin_volume_acc = ncomb(c.fin_volume_acc, tfv);
    if (logl) c.leaf_count += c.s - c.n_surv;
    c.s = 2 * c.n_surv;
    c.it += 1;
  }
  __threadfence();
}

// ------------------------------------------------------- FP64 peak probe
__global__ void k_fp64_calls(double* out, int iters, int which) {
  double x = 1e-3 * (threadIdx.x + 1), s = 0.0, c = 0.0;
  for (int it = 0; it < iters; ++it) {
    if (which == 0) {
      s += exp(-x);
    } else if (which == 1) {
      double sn, cs;
      sincos(x, &sn, &cs);
      s += sn;
      c += cs;
    } else {
      s += 1.0 / x;
    }
    x += 1e-7;
  }
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s + c;
}

__global__ void k_fp64_fma(double* out, int iters, double a, double b) {
  double x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = threadIdx.x * 1e-3 + i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = fma(x[i], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += x[i];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// --------------------------------------------------------------- workspace
struct GraphEntry {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

struct Workspace {
  int dev = -1;
  int sms = 0;
  int64_t cap = 0;
  int n = 0;
  Pool pool = {};
  Ctrl* ctrl = nullptr;
  IntegrandParams* prm = nullptr;
  EvalPartial* eval_part = nullptr;
  ProbeAcc* probe_acc = nullptr;  // kProbeBins bins, zero between probe passes
  CountPartial* count_part = nullptr;
  TraceRec* trace = nullptr;
  int trace_cap = 0;
  void* fcache = nullptr;
  LeafLog leaves = {nullptr, nullptr, 0};
  void* leaf_alloc[2] = {nullptr, nullptr};
  int leaf_n = 0;
  int64_t last_leaves = -1;   // leaf count of the last integration that kept them
  uint64_t* codes[kMaxDim + 1] = {nullptr};
  int ncodes[kMaxDim + 1] = {0};
  double* grad_terms = nullptr;  // per-axis chain-rule terms of the cached intervals
  double* grad_part = nullptr;
  unsigned int* grad_ticket = nullptr;
  double* grad_out = nullptr;
  int max_grid = 0;
  cudaStream_t own_stream = nullptr;
  std::vector<void*> allocs;
  std::map<int, GraphEntry> graphs;  // key = family * 16 + dim
};

static std::mutex g_mu;
static Workspace g_ws;
static std::map<int, RuleTable> g_rules;

constexpr int kMgmtThreads = 256;
constexpr int kMgmtItems = 8;
constexpr int kTraceCap = 1024;

static const FamilyKernels& family_kernels(int fam, int degree = 9) {
  if (degree == 7) {
    switch (fam) {
      case kFamProductPeak: return kernels_product_peak_gm7();
      case kFamGaussian: return kernels_gaussian_gm7();
      case kFamOscillatory: return kernels_oscillatory_gm7();
      case kFamCornerPeak: return kernels_corner_peak_gm7();
      case kFamDiscontinuous: return kernels_discontinuous_gm7();
      case kFamBoxPower: return kernels_box_power_gm7();
      default: return kernels_c0_gm7();
    }
  }
  switch (fam) {
    case kFamProductPeak: return kernels_product_peak();
    case kFamGaussian: return kernels_gaussian();
    case kFamOscillatory: return kernels_oscillatory();
    case kFamCornerPeak: return kernels_corner_peak();
    case kFamDiscontinuous: return kernels_discontinuous();
    case kFamBoxPower: return kernels_box_power();
    default: return kernels_c0();
  }
}

// The rule degree of an options value: 0 or 9 the degree-9 rule, 7 the
// Genz-Malik variant, anything else -1.
static int rule_degree(int32_t v) { return (v == 0 || v == 9) ? 9 : v == 7 ? 7 : -1; }

static void release_graphs(Workspace& w) {
  for (auto& kv : w.graphs) {
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
  }
  w.graphs.clear();
}

static void release_leaf_log(Workspace& w) {
  for (void*& p : w.leaf_alloc) {
    if (p) cudaFree(p);
    p = nullptr;
  }
  w.leaves = LeafLog{nullptr, nullptr, 0};
  w.leaf_n = 0;
  w.last_leaves = -1;
}

static void release_ws(Workspace& w) {
  release_graphs(w);
  release_leaf_log(w);
  for (void* p : w.allocs) cudaFree(p);
  w.allocs.clear();
  for (int i = 0; i <= kMaxDim; ++i) {
    w.codes[i] = nullptr;
    w.ncodes[i] = 0;
  }
  w.cap = 0;
  w.n = 0;
  w.pool = Pool{};
  w.ctrl = nullptr;
}

template <class T>
static cudaError_t ws_alloc(Workspace& w, T** p, size_t count) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, count * sizeof(T) + 256);
  if (e != cudaSuccess) return e;
  w.allocs.push_back(q);
  *p = reinterpret_cast<T*>(q);
  return cudaSuccess;
}

static int ensure_workspace(int64_t want_cap, int n) {
  Workspace& w = g_ws;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(PAGANI_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (w.dev == dev && w.cap >= want_cap && w.n >= n) return 0;
  release_ws(w);
  w.dev = dev;
  cudaDeviceGetAttribute(&w.sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t cap = ((want_cap + 4095) / 4096) * 4096;
  const int nn = n;
  w.max_grid = w.sms * 16;
  const int64_t ntiles = cap / kTile + 2;
#define PG_ALLOC(ptr, cnt)                                                                        \
  do {                                                                                            \
    e = ws_alloc(w, &(ptr), (size_t)(cnt));                                                       \
    if (e != cudaSuccess) {                                                                       \
      release_ws(w);                                                                              \
      return fail(PAGANI_ERR_CUDA, std::string("workspace allocation: ") + cudaGetErrorString(e)); \
    }                                                                                             \
  } while (0)
  PG_ALLOC(w.pool.lower, (size_t)2 * nn * cap);
  PG_ALLOC(w.pool.level, (size_t)2 * nn * cap);
  PG_ALLOC(w.pool.V, cap);
  PG_ALLOC(w.pool.E, cap);
  PG_ALLOC(w.pool.K, cap);
  PG_ALLOC(w.pool.act, cap);
  PG_ALLOC(w.pool.Vp, cap / 2 + 1);
  PG_ALLOC(w.pool.tile_count, ntiles * kTileWarps);
  PG_ALLOC(w.pool.tile_offset, ntiles);
  PG_ALLOC(w.ctrl, 1);
  PG_ALLOC(w.prm, 1);
  PG_ALLOC(w.eval_part, w.max_grid);
  PG_ALLOC(w.probe_acc, kProbeBins);
  PG_ALLOC(w.count_part, w.max_grid);
  PG_ALLOC(w.trace, kTraceCap);
  {
    double2* fc = nullptr;  // sized for the widest element type (complex factors)
    PG_ALLOC(fc, (size_t)kMaxDim * kCacheSlots * kCodes);
    w.fcache = fc;
  }
  PG_ALLOC(w.grad_terms, (size_t)kMaxDim * kCacheSlots * kGradTerms);
  PG_ALLOC(w.grad_part, (size_t)w.max_grid * (2 * kMaxDim + 1) * 2);
  PG_ALLOC(w.grad_ticket, 1);
  PG_ALLOC(w.grad_out, 2 * kMaxDim + 1);
  for (int d = 2; d <= kMaxDim; ++d) {
    std::vector<uint64_t> pc = point_codes(d);
    PG_ALLOC(w.codes[d], pc.size());
    w.ncodes[d] = (int)pc.size();
    e = cudaMemcpy(w.codes[d], pc.data(), pc.size() * sizeof(uint64_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail(PAGANI_ERR_CUDA, cudaGetErrorString(e));
  }
  e = cudaMemset(w.grad_ticket, 0, sizeof(unsigned int));
  if (e != cudaSuccess) return fail(PAGANI_ERR_CUDA, cudaGetErrorString(e));
#undef PG_ALLOC
  w.pool.cap = cap;
  w.pool.n = nn;
  w.cap = cap;
  w.n = nn;
  w.trace_cap = kTraceCap;
  e = cudaMemset(w.ctrl, 0, sizeof(Ctrl));
  if (e != cudaSuccess) return fail(PAGANI_ERR_CUDA, cudaGetErrorString(e));
  if (!w.own_stream) cudaStreamCreateWithFlags(&w.own_stream, cudaStreamNonBlocking);
  return 0;
}

// Leaf log for up to cap boxes of dimension n (allocated on first request;
// the cached graphs embed its pointers, so they are rebuilt when it moves).
static int ensure_leaf_log(int64_t cap, int n) {
  Workspace& w = g_ws;
  if (w.leaves.lower && w.leaves.cap >= cap && w.leaf_n >= n) return 0;
  release_graphs(w);
  release_leaf_log(w);
  cudaError_t e = cudaMalloc(&w.leaf_alloc[0], sizeof(double) * (size_t)n * cap);
  if (e == cudaSuccess) e = cudaMalloc(&w.leaf_alloc[1], (size_t)n * cap);
  if (e != cudaSuccess) {
    release_leaf_log(w);
    return fail(PAGANI_ERR_CUDA, std::string("leaf log allocation: ") + cudaGetErrorString(e));
  }
  w.leaves.lower = static_cast<double*>(w.leaf_alloc[0]);
  w.leaves.level = static_cast<uint8_t*>(w.leaf_alloc[1]);
  w.leaves.cap = cap;
  w.leaf_n = n;
  return 0;
}

static const RuleTable* get_rule(int n, int degree = 9) {
  const int key = n * 16 + degree;
  auto it = g_rules.find(key);
  if (it != g_rules.end()) return &it->second;
  RuleTable t;
  double res = 0.0;
  if (!build_rule(n, degree, &t, &res) || !(res < 1e-14)) return nullptr;
  return &(g_rules[key] = t);
}

static EvalRule to_eval_rule(const RuleTable& t) {
  EvalRule r;
  for (int i = 0; i < 5; ++i) r.radius[i] = t.radius[i];
  r.q = t.q;
  r.q_outer = t.q_outer;
  r.noise = 64.0 * (double)t.num_points * 0x1p-53;
  for (int g = 0; g < kNumGen; ++g) r.cnt[g] = (double)t.count[g];
  for (int k = 0; k < 4; ++k) {
    r.umax[k] = 0.0;
    r.floor_unit[k] = 0.0;
    for (int g = 0; g < kNumGen; ++g) {
      r.umax[k] = std::fmax(r.umax[k], std::fabs(t.w[g][1 + k]));
      r.floor_unit[k] = std::fma(std::fabs(t.w[g][1 + k]), (double)t.count[g], r.floor_unit[k]);
    }
  }
  for (int g = 0; g < kNumGen; ++g)
    for (int k = 0; k < 5; ++k) r.w[g][k] = t.w[g][k];
  r.vround_unit = 0.0;
  for (int g = 0; g < kNumGen; ++g) r.vround_unit = std::fma(std::fabs(t.w[g][0]), (double)t.count[g], r.vround_unit);
  return r;
}

static int param_count(int fam, int n) {
  switch (fam) {
    case kFamOscillatory: return n + 1;
    case kFamCornerPeak: return n;
    case kFamBoxPower: return 1;
    default: return 2 * n;
  }
}

static int check_params(int fam, int n, const double* p) {
  const int np = param_count(fam, n);
  for (int i = 0; i < np; ++i)
    if (!std::isfinite(p[i])) return fail(PAGANI_ERR_INTEGRAND, "non-finite integrand parameter");
  if (fam == kFamProductPeak)
    for (int j = 0; j < n; ++j)
      if (p[j] == 0.0) return fail(PAGANI_ERR_INTEGRAND, "product peak needs c_j != 0");
  if (fam == kFamBoxPower && p[0] < 0.0) return fail(PAGANI_ERR_INTEGRAND, "box power needs q >= 0");
  return 0;
}

static IntegrandParams to_params(int fam, int n, const double* p) {
  IntegrandParams q;
  std::memset(&q, 0, sizeof(q));
  for (int j = 0; j < kMaxDim; ++j) q.len[j] = 1.0;  // the unit cube
  q.vol = 1.0;
  if (fam == kFamOscillatory) {
    q.u = p[0];
    for (int j = 0; j < n; ++j) q.p0[j] = p[1 + j];
  } else if (fam == kFamBoxPower) {
    q.u = p[0];
  } else if (fam == kFamCornerPeak) {
    for (int j = 0; j < n; ++j) q.p0[j] = p[j];
  } else {
    for (int j = 0; j < n; ++j) {
      q.p0[j] = p[j];
      q.p1[j] = p[n + j];
    }
  }
  return q;
}

// Threshold-Classify triggers of an options value: bit 0 the estimate's
// digits unchanged, bit 1 memory about to be exhausted (Sec. 3.5.2).
static int32_t trigger_mask(int32_t heuristic_filter) {
  switch (heuristic_filter) {
    case 0: return 0;
    case 2: return 2;
    case 3: return 1;
    default: return 3;
  }
}

static int default_init_div(int n) {
  int d = 2;
  for (;;) {
    int64_t pw = 1;
    for (int j = 0; j < n; ++j) pw *= 2 * d;
    if (pw > 4096) break;
    d *= 2;
  }
  return d;
}

struct Launch {
  int eval_grid, eval_block;
  size_t eval_smem;
  int mgmt_grid;
  int probe_grid;
  int count_grid;
};

static int launch_config(const FamilyKernels& fk, int n, Launch* L) {
  Workspace& w = g_ws;
  L->eval_block = fk.threads;
  L->eval_smem = (size_t)fk.table_bytes_per_thread[n] * fk.threads;
  int occ = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fk.loop_fn[n], fk.threads, L->eval_smem);
  if (e != cudaSuccess || occ < 1)
    return fail(PAGANI_ERR_CUDA, std::string("evaluate kernel does not fit: ") + cudaGetErrorString(e));
  L->eval_grid = w.sms * occ;
  if (L->eval_grid > w.max_grid) L->eval_grid = w.max_grid;
  L->mgmt_grid = w.sms * 2;
  if (L->mgmt_grid > w.max_grid) L->mgmt_grid = w.max_grid;
  L->probe_grid = w.sms * 5;
  if (L->probe_grid > w.max_grid) L->probe_grid = w.max_grid;
  L->count_grid = w.sms * 4;
  if (L->count_grid > w.max_grid) L->count_grid = w.max_grid;
  return 0;
}

static LoopArgs loop_args(int n, int use_graph, cudaGraphConditionalHandle hm, cudaGraphConditionalHandle hp) {
  Workspace& w = g_ws;
  LoopArgs a;
  std::memset(&a, 0, sizeof(a));
  a.codes = w.codes[n];
  a.gen_off[0] = 0;
  for (int g = 0; g < kNumGen; ++g) a.gen_off[g + 1] = a.gen_off[g] + (int)orbit_count(n, g);
  a.pool = w.pool;
  a.ctrl = w.ctrl;
  a.prm = w.prm;
  a.eval_part = w.eval_part;
  a.probe_acc = w.probe_acc;
  a.count_part = w.count_part;
  a.trace = w.trace;
  a.trace_cap = w.trace_cap;
  a.use_graph = use_graph;
  a.h_main = hm;
  a.h_probe = hp;
  a.fcache = w.fcache;
  a.fcache_levels = kCacheLevels;
  a.leaves = w.leaves;
  return a;
}

static cudaError_t add_kernel(cudaGraphNode_t* node, cudaGraph_t g, const cudaGraphNode_t* dep, size_t ndep,
                              const void* fn, int grid, int block, size_t smem, void** args) {
  cudaKernelNodeParams kp;
  std::memset(&kp, 0, sizeof(kp));
  kp.func = const_cast<void*>(fn);
  kp.gridDim = dim3(grid);
  kp.blockDim = dim3(block);
  kp.sharedMemBytes = (unsigned)smem;
  kp.kernelParams = args;
  return cudaGraphAddKernelNode(node, g, dep, ndep, &kp);
}

static cudaError_t add_while(cudaGraphNode_t* node, cudaGraph_t g, const cudaGraphNode_t* dep, size_t ndep,
                             cudaGraphConditionalHandle h, cudaGraph_t* body) {
  alignas(cudaGraphNodeParams) unsigned char raw[sizeof(cudaGraphNodeParams)];
  std::memset(raw, 0, sizeof(raw));
  cudaGraphNodeParams& np = *reinterpret_cast<cudaGraphNodeParams*>(raw);
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaError_t e = cudaGraphAddNode(node, g, dep, nullptr, ndep, &np);
  if (e == cudaSuccess) *body = np.conditional.phGraph_out[0];
  return e;
}

// The whole iteration loop of Algorithm 2 as one graph:
//   WHILE(main) { evaluate -> WHILE(probe) { probe } -> count -> split }
static int build_graph(int fam, int n, int degree, const EvalRule& rule, const Launch& L, GraphEntry* out) {
  const FamilyKernels& fk = family_kernels(fam, degree);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaGraphCreate(&g, 0);
  if (e != cudaSuccess) return fail(PAGANI_ERR_CUDA, std::string("cudaGraphCreate: ") + cudaGetErrorString(e));
  cudaGraphConditionalHandle hm, hp;
  cudaGraphNode_t wmain, nev, wprobe, nprobe, ncount, nsplit;  // and the cache fill
  cudaGraph_t body = nullptr, pbody = nullptr;
  LoopArgs args;
  EvalRule r = rule;
  void* eargs[2];
  void* margs[1];
#define PG_CK(x)                                                                     \
  do {                                                                               \
    e = (x);                                                                         \
    if (e != cudaSuccess) {                                                          \
      cudaGraphDestroy(g);                                                           \
      return fail(PAGANI_ERR_CUDA, std::string(#x ": ") + cudaGetErrorString(e));    \
    }                                                                                \
  } while (0)
  PG_CK(cudaGraphConditionalHandleCreate(&hm, g, 1, cudaGraphCondAssignDefault));
  // the factor cache is filled once, ahead of the loop
  cudaGraphNode_t nfill;
  args = loop_args(n, 1, hm, 0);
  eargs[0] = &r;
  eargs[1] = &args;
  margs[0] = &args;
  PG_CK(add_kernel(&nfill, g, nullptr, 0, fk.fill_fn[n], L.mgmt_grid, 256, 0, eargs));
  PG_CK(add_while(&wmain, g, &nfill, 1, hm, &body));
  PG_CK(cudaGraphConditionalHandleCreate(&hp, body, 0, 0));
  args = loop_args(n, 1, hm, hp);
  PG_CK(add_kernel(&nev, body, nullptr, 0, fk.loop_fn[n], L.eval_grid, L.eval_block, L.eval_smem, eargs));
  PG_CK(add_while(&wprobe, body, &nev, 1, hp, &pbody));
  PG_CK(add_kernel(&nprobe, pbody, nullptr, 0, (const void*)&k_probe<kProbeThreads>, L.probe_grid, kProbeThreads,
                   0, margs));
  PG_CK(add_kernel(&ncount, body, &wprobe, 1, (const void*)&k_count<kMgmtThreads, kMgmtItems>, L.count_grid,
                   kMgmtThreads, 0, margs));
  PG_CK(add_kernel(&nsplit, body, &ncount, 1, (const void*)&k_split<kMgmtThreads, kMgmtItems>, L.mgmt_grid,
                   kMgmtThreads, 0, margs));
  cudaGraphExec_t ex = nullptr;
  PG_CK(cudaGraphInstantiate(&ex, g, 0));
#undef PG_CK
  out->graph = g;
  out->exec = ex;
  return 0;
}

static int integrate_locked(int n, int fam, const double* params, const double* lower, const double* upper,
                            double epsrel, double epsabs, int64_t max_regions, const pagani_options& o,
                            cudaStream_t st, pagani_result* out, pagani_trace_record* trace, int trace_cap) {
  std::memset(out, 0, sizeof(*out));
  if (n < PAGANI_MIN_DIM || n > PAGANI_MAX_DIM) return out->status = fail(PAGANI_ERR_DIM, "dim must be in [2, 8]");
  if (fam < 0 || fam >= kNumFamilies) return out->status = fail(PAGANI_ERR_INTEGRAND, "unknown integrand_id");
  if (!params) return out->status = fail(PAGANI_ERR_ARGUMENT, "params is NULL");
  if (!(epsrel > 0.0) || !(epsabs >= 0.0) || !std::isfinite(epsrel) || !std::isfinite(epsabs))
    return out->status = fail(PAGANI_ERR_TOLERANCE, "need epsrel > 0 and epsabs >= 0, finite");
  if (o.it_max < 1 || o.it_max > kTraceCap) return out->status = fail(PAGANI_ERR_ARGUMENT, "it_max out of range");
  if (o.heuristic_filter < 0 || o.heuristic_filter > 3)
    return out->status = fail(PAGANI_ERR_ARGUMENT, "heuristic_filter must be 0..3");
  const int deg = rule_degree(o.rule_degree);
  if (deg < 0) return out->status = fail(PAGANI_ERR_ARGUMENT, "rule_degree must be 9 (or 0) or 7");
  if (deg != 9 && o.keep_leaves)
    return out->status = fail(PAGANI_ERR_ARGUMENT, "keep_leaves (differentiation) needs the degree-9 rule");
  int rc = check_params(fam, n, params);
  if (rc) return out->status = rc;
  if ((lower == nullptr) != (upper == nullptr))
    return out->status = fail(PAGANI_ERR_ARGUMENT, "give both bounds or neither");
  double bound_vol = 1.0;
  for (int j = 0; lower && j < n; ++j) {
    const double len = upper[j] - lower[j];
    if (!std::isfinite(lower[j]) || !std::isfinite(upper[j]) || !(len > 0.0) || !std::isfinite(len))
      return out->status = fail(PAGANI_ERR_ARGUMENT, "bounds must be finite with upper > lower");
    bound_vol *= len;
  }
  if (!(bound_vol > 0.0) || !std::isfinite(bound_vol))
    return out->status = fail(PAGANI_ERR_ARGUMENT, "the volume of the bounds is not a normal number");
  const int d0 = o.init_div > 0 ? o.init_div : default_init_div(n);
  int log2d = 0;
  while ((1 << log2d) < d0) ++log2d;
  if ((1 << log2d) != d0 || log2d > 20) return out->status = fail(PAGANI_ERR_ARGUMENT, "init_div must be a power of two");
  int64_t s0 = 1;
  for (int j = 0; j < n; ++j) {
    s0 *= d0;
    if (s0 > ((int64_t)1 << 40)) return out->status = fail(PAGANI_ERR_ARGUMENT, "initial split too large");
  }
  if (s0 > max_regions) return out->status = fail(PAGANI_ERR_CAPACITY, "max_regions below the initial split");
  const RuleTable* rt = get_rule(n, deg);
  if (!rt) return out->status = fail(PAGANI_ERR_CUDA, "rule construction failed");
  rc = ensure_workspace(max_regions > s0 ? max_regions : s0, n);
  if (rc) return out->status = rc;
  Workspace& w = g_ws;
  if (o.keep_leaves) {
    rc = ensure_leaf_log(4 * (max_regions > s0 ? max_regions : s0), n);
    if (rc) return out->status = rc;
  }
  w.last_leaves = -1;
  if (!st) st = w.own_stream;
  const FamilyKernels& fk = family_kernels(fam, deg);
  Launch L;
  rc = launch_config(fk, n, &L);
  if (rc) return out->status = rc;
  const EvalRule rule = to_eval_rule(*rt);

  Ctrl h;
  std::memset(&h, 0, sizeof(h));
  h.tau_rel = epsrel;
  h.tau_cls = epsrel;
  h.tau_abs = epsabs;
  h.max_regions = max_regions;
  h.it_max = o.it_max;
  h.relerr_filter = o.relerr_filter ? 1 : 0;
  h.heuristic_filter = trigger_mask(o.heuristic_filter);
  h.trace_on = trace != nullptr ? 1 : 0;
  h.s = s0;
  h.it = 1;
  h.status = -100;
  h.l0 = log2d;
  h.keep_leaves = o.keep_leaves ? 1 : 0;
  IntegrandParams prm = to_params(fam, n, params);
  if (lower) {
    for (int j = 0; j < n; ++j) {
      prm.lo[j] = lower[j];
      prm.len[j] = upper[j] - lower[j];
    }
    prm.vol = bound_vol;
  }
  cudaError_t e;
#define PG_CK(x)                                                                          \
  do {                                                                                    \
    e = (x);                                                                              \
    if (e != cudaSuccess) return out->status = fail(PAGANI_ERR_CUDA, std::string(#x ": ") + cudaGetErrorString(e)); \
  } while (0)
  // the pool must be indexed with the call's dimension
  w.pool.n = n;
  PG_CK(cudaMemcpyAsync(w.ctrl, &h, sizeof(Ctrl), cudaMemcpyHostToDevice, st));
  PG_CK(cudaMemsetAsync(w.probe_acc, 0, sizeof(ProbeAcc) * kProbeBins, st));  // probe bins start at zero
  PG_CK(cudaMemcpyAsync(w.prm, &prm, sizeof(prm), cudaMemcpyHostToDevice, st));
  {
    Pool p = w.pool;
    k_uniform_split<<<(int)((s0 + 255) / 256), 256, 0, st>>>(p, d0, log2d, s0);
    PG_CK(cudaGetLastError());
  }
  int64_t h2d = sizeof(Ctrl) + sizeof(prm), d2h = 0;
  int launches = 1, eval_launches = 0;  // the Uniform-Split kernel
  out->eval_ms = -1.0;
  for (int i = 0; i < 4; ++i) out->phase_ms[i] = -1.0;
  if (o.use_graph) {
    const int key = fam * 16 + n + (w.n << 8) + (deg << 16);
    auto it = w.graphs.find(key);
    if (it == w.graphs.end()) {
      GraphEntry ge;
      rc = build_graph(fam, n, deg, rule, L, &ge);
      if (rc) return out->status = rc;
      it = w.graphs.emplace(key, ge).first;
    }
    PG_CK(cudaGraphLaunch(it->second.exec, st));
    PG_CK(cudaMemcpyAsync(&h, w.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
    PG_CK(cudaStreamSynchronize(st));
    d2h += sizeof(Ctrl);
  } else {
    // host-driven loop: the same kernels, one launch each, with CUDA events
    // around every Evaluate launch on the launching stream
    // host-driven loop: the same kernels, one launch each, with CUDA events
    // around every launch on the launching stream (the per-phase breakdown)
    const LoopArgs args = loop_args(n, 0, 0, 0);
    cudaEvent_t ev[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    for (int i = 0; i < 6; ++i) PG_CK(cudaEventCreate(&ev[i]));
    double eval_ms = 0.0, phase[4] = {0.0, 0.0, 0.0, 0.0};
    auto elapsed = [&](cudaEvent_t a, cudaEvent_t b) {
      float ms = 0.f;
      return cudaEventElapsedTime(&ms, a, b) == cudaSuccess ? (double)ms : 0.0;
    };
    PG_CK(cudaEventRecord(ev[0], st));
    PG_CK(fk.fill[n](rule, args, L.mgmt_grid, 256, 0, st));  // the factor cache, once
    PG_CK(cudaEventRecord(ev[1], st));
    ++launches;
    PG_CK(cudaEventSynchronize(ev[1]));
    phase[0] += elapsed(ev[0], ev[1]);
    for (int guard = 0; guard < o.it_max + 2; ++guard) {
      PG_CK(cudaEventRecord(ev[1], st));
      PG_CK(fk.loop[n](rule, args, L.eval_grid, L.eval_block, L.eval_smem, st));
      PG_CK(cudaEventRecord(ev[2], st));
      ++launches;
      PG_CK(cudaMemcpyAsync(&h, w.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
      PG_CK(cudaStreamSynchronize(st));
      d2h += sizeof(Ctrl);
      eval_ms += elapsed(ev[1], ev[2]);
      ++eval_launches;
      if (h.search) {
        for (int probe = 0; probe < 128; ++probe) {
          PG_CK(cudaEventRecord(ev[0], st));
          k_probe<kProbeThreads><<<L.probe_grid, kProbeThreads, 0, st>>>(args);
          PG_CK(cudaGetLastError());
          PG_CK(cudaEventRecord(ev[1], st));
          ++launches;
          PG_CK(cudaMemcpyAsync(&h, w.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
          PG_CK(cudaStreamSynchronize(st));
          d2h += sizeof(Ctrl);
          phase[1] += elapsed(ev[0], ev[1]);
          if (!h.search_cont) break;
        }
      }
      PG_CK(cudaEventRecord(ev[3], st));
      k_count<kMgmtThreads, kMgmtItems><<<L.count_grid, kMgmtThreads, 0, st>>>(args);
      PG_CK(cudaGetLastError());
      PG_CK(cudaEventRecord(ev[4], st));
      k_split<kMgmtThreads, kMgmtItems><<<L.mgmt_grid, kMgmtThreads, 0, st>>>(args);
      PG_CK(cudaGetLastError());
      PG_CK(cudaEventRecord(ev[5], st));
      launches += 2;
      PG_CK(cudaMemcpyAsync(&h, w.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
      PG_CK(cudaStreamSynchronize(st));
      d2h += sizeof(Ctrl);
      phase[2] += elapsed(ev[3], ev[4]);
      phase[3] += elapsed(ev[4], ev[5]);
      if (h.done) break;
    }
    for (int i = 0; i < 6; ++i) cudaEventDestroy(ev[i]);
    out->eval_ms = eval_ms;
    for (int i = 0; i < 4; ++i) out->phase_ms[i] = phase[i];
  }
  if (trace && trace_cap > 0) {
    const int nrec = std::min(std::min(h.it, trace_cap), w.trace_cap);
    if (nrec > 0) {
      std::vector<TraceRec> tmp(nrec);
      PG_CK(cudaMemcpyAsync(tmp.data(), w.trace, sizeof(TraceRec) * nrec, cudaMemcpyDeviceToHost, st));
      PG_CK(cudaStreamSynchronize(st));
      static_assert(sizeof(TraceRec) == sizeof(pagani_trace_record), "trace layout");
      std::memcpy(trace, tmp.data(), sizeof(TraceRec) * nrec);
      d2h += (int64_t)sizeof(TraceRec) * nrec;
    }
  }
#undef PG_CK
  if (o.use_graph) {
    // the graph ran the cache fill once, then one Evaluate, count and split
    // per iteration plus the probes
    eval_launches = h.it;
    launches += 1 + 3 * h.it + h.total_passes;
  }
  out->eval_launches = eval_launches;
  out->kernel_launches = launches;
  out->h2d_bytes = h2d;
  out->d2h_bytes = d2h;
  out->estimate = h.estimate;
  out->errorest = h.errorest;
  out->iterations = h.it;
  out->n_regions = h.n_regions_total;
  out->n_active_last = h.s;
  // the device tracks volumes of the unit cube; report them on the bounds
  out->finished_volume = nval(h.fin_volume_acc) * bound_vol;
  out->active_volume = h.active_volume * bound_vol;
  out->n_leaves = -1;
  if (o.keep_leaves && h.done) {
    if (h.leaf_overflow) {
      g_err = "the leaf log ran out of room; n_leaves = -1";
    } else {
      out->n_leaves = h.leaf_count + h.s;
      w.last_leaves = out->n_leaves;
      w.leaf_n = n;
    }
  }
  if (h.watchdog == 1) return out->status = fail(PAGANI_ERR_WATCHDOG, "region depth limit reached on one axis");
  if (h.watchdog == 3) return out->status = fail(PAGANI_ERR_WATCHDOG, "threshold search left its probe tree");
  if (h.watchdog) return out->status = fail(PAGANI_ERR_WATCHDOG, "device loop exceeded its iteration bound");
  if (!h.done) return out->status = fail(PAGANI_ERR_WATCHDOG, "device loop ended without a result");
  out->status = h.status;
  if (h.status == -6) g_err = "the integrand produced NaN or Inf";
  return out->status;
}

// ------------------------------------------------------ allocation-free path
// Some callers cannot call cudaMalloc: applications whose own allocator owns
// all device memory, or latency-critical service loops that must never
// allocate.  pagani_integrate_noalloc serves them: it runs the same loop
// kernels on scratch memory carved from this file-scope array instead of the
// library workspace.  Every GPU that loads the library holds the array until
// the process exits.
constexpr size_t kNoallocBytes = (size_t)32 << 20;  // 32 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

// Host code may not use g_noalloc_scratch directly (its host-side name is a
// stand-in, not a device address); this is the device address per device,
// looked up once with that device current.
static void* g_noalloc_base[64] = {nullptr};

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct NoallocLayout {
  size_t ctrl, prm, eval_part, probe_acc, count_part, lower, level, V, E, K, act, Vp, tile_count, tile_offset, total;
};

static NoallocLayout noalloc_layout(int64_t cap, int n, int max_grid) {
  NoallocLayout L;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t at = off;
    off = align256(off + bytes);
    return at;
  };
  const int64_t ntiles = cap / kTile + 2;
  L.ctrl = take(sizeof(Ctrl));
  L.prm = take(sizeof(IntegrandParams));
  L.eval_part = take(sizeof(EvalPartial) * (size_t)max_grid);
  L.probe_acc = take(sizeof(ProbeAcc) * (size_t)kProbeBins);
  L.count_part = take(sizeof(CountPartial) * (size_t)max_grid);
  L.lower = take(sizeof(double) * 2 * (size_t)n * cap);
  L.level = take((size_t)2 * n * cap);
  L.V = take(sizeof(double) * (size_t)cap);
  L.E = take(sizeof(double) * (size_t)cap);
  L.K = take((size_t)cap);
  L.act = take((size_t)cap);
  L.Vp = take(sizeof(double) * (size_t)(cap / 2 + 1));
  L.tile_count = take(sizeof(int) * (size_t)ntiles * kTileWarps);
  L.tile_offset = take(sizeof(long long) * (size_t)ntiles);
  L.total = off;
  return L;
}

// Largest region capacity (a multiple of 4096) whose layout fits the array.
// A region takes 18n + 22 bytes of the layout plus its share of the tile
// arrays, so kNoallocBytes / (18n + 22) bounds the capacity from above.
static int64_t noalloc_capacity(int n, int max_grid) {
  int64_t lo = 0, hi = (int64_t)(kNoallocBytes / (size_t)(18 * n + 22)) + 4096;
  while (hi - lo > 4096) {
    const int64_t mid = ((lo + hi) / 2 / 4096) * 4096;
    if (mid <= lo) break;
    if (noalloc_layout(mid, n, max_grid).total <= kNoallocBytes) lo = mid;
    else hi = mid;
  }
  return lo;
}

static int integrate_noalloc_locked(int n, int fam, const double* params, double epsrel, double epsabs,
                                    int64_t max_regions, cudaStream_t st, pagani_result* out) {
  std::memset(out, 0, sizeof(*out));
  out->eval_ms = -1.0;
  for (int k = 0; k < 4; ++k) out->phase_ms[k] = -1.0;
  if (n < PAGANI_MIN_DIM || n > PAGANI_MAX_DIM) return out->status = fail(PAGANI_ERR_DIM, "dim must be in [2, 8]");
  if (fam < 0 || fam >= kNumFamilies) return out->status = fail(PAGANI_ERR_INTEGRAND, "unknown integrand_id");
  if (!params) return out->status = fail(PAGANI_ERR_ARGUMENT, "params is NULL");
  if (!(epsrel > 0.0) || !(epsabs >= 0.0) || !std::isfinite(epsrel) || !std::isfinite(epsabs))
    return out->status = fail(PAGANI_ERR_TOLERANCE, "need epsrel > 0 and epsabs >= 0, finite");
  int rc = check_params(fam, n, params);
  if (rc) return out->status = rc;
  const int d0 = default_init_div(n);
  int log2d = 0;
  while ((1 << log2d) < d0) ++log2d;
  int64_t s0 = 1;
  for (int j = 0; j < n; ++j) s0 *= d0;
  if (s0 > max_regions) return out->status = fail(PAGANI_ERR_CAPACITY, "max_regions below the initial split");
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 64)
    return out->status = fail(PAGANI_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int max_grid = sms * 16;
  const int64_t cap_max = noalloc_capacity(n, max_grid);
  if (max_regions > cap_max)
    return out->status = fail(PAGANI_ERR_CAPACITY,
                              "max_regions " + std::to_string(max_regions) + " exceeds the allocation-free capacity " +
                                  std::to_string(cap_max) + " regions for dim " + std::to_string(n) +
                                  " (32 MiB static scratch)");
  if (!g_noalloc_base[dev]) {
    // set-up, once per device, with that device current
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || !ptr)
      return out->status = fail(PAGANI_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_noalloc_base[dev] = ptr;
  }
  unsigned char* base = static_cast<unsigned char*>(g_noalloc_base[dev]);
  const RuleTable* rt = get_rule(n);
  if (!rt) return out->status = fail(PAGANI_ERR_CUDA, "rule construction failed");
  const FamilyKernels& fk = family_kernels(fam);
  // launch shape as in the workspace path
  Launch Lc;
  Lc.eval_block = fk.threads;
  Lc.eval_smem = (size_t)fk.table_bytes_per_thread[n] * fk.threads;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fk.loop_fn[n], fk.threads, Lc.eval_smem);
  if (e != cudaSuccess || occ < 1) return out->status = fail(PAGANI_ERR_CUDA, "evaluate kernel does not fit");
  Lc.eval_grid = sms * occ < max_grid ? sms * occ : max_grid;
  Lc.mgmt_grid = sms * 2;
  Lc.probe_grid = sms * 5;
  Lc.count_grid = sms * 4;
  const int64_t cap = ((max_regions + 4095) / 4096) * 4096;
  const NoallocLayout L = noalloc_layout(cap, n, max_grid);
  LoopArgs a;
  std::memset(&a, 0, sizeof(a));
  a.pool.lower = reinterpret_cast<double*>(base + L.lower);
  a.pool.level = base + L.level;
  a.pool.V = reinterpret_cast<double*>(base + L.V);
  a.pool.E = reinterpret_cast<double*>(base + L.E);
  a.pool.K = base + L.K;
  a.pool.act = base + L.act;
  a.pool.Vp = reinterpret_cast<double*>(base + L.Vp);
  a.pool.tile_count = reinterpret_cast<int*>(base + L.tile_count);
  a.pool.tile_offset = reinterpret_cast<long long*>(base + L.tile_offset);
  a.pool.cap = cap;
  a.pool.n = n;
  a.ctrl = reinterpret_cast<Ctrl*>(base + L.ctrl);
  a.prm = reinterpret_cast<const IntegrandParams*>(base + L.prm);
  a.eval_part = reinterpret_cast<EvalPartial*>(base + L.eval_part);
  a.probe_acc = reinterpret_cast<ProbeAcc*>(base + L.probe_acc);
  a.count_part = reinterpret_cast<CountPartial*>(base + L.count_part);
  a.trace = nullptr;
  a.trace_cap = 0;
  a.use_graph = 0;
  // every call starts from a fully written control block (tickets, sums and
  // counters at zero) and parameter block; the pool, partials and tile
  // arrays are written before they are read, so stale contents of the
  // previous call do not matter
  Ctrl h;
  std::memset(&h, 0, sizeof(h));
  h.tau_rel = epsrel;
  h.tau_cls = epsrel;
  h.tau_abs = epsabs;
  h.max_regions = max_regions;
  h.it_max = 100;
  h.relerr_filter = fam == kFamOscillatory ? 0 : 1;
  h.heuristic_filter = trigger_mask(1);
  h.s = s0;
  h.it = 1;
  h.status = -100;
  IntegrandParams prm = to_params(fam, n, params);
  const EvalRule rule = to_eval_rule(*rt);
  // on an error, wait for the work already queued on st before returning:
  // no kernel of a failed call may still write the shared array when the
  // next call (perhaps on another stream) starts rewriting it
#define PG_CK(x)                                                                          \
  do {                                                                                    \
    e = (x);                                                                              \
    if (e != cudaSuccess) {                                                               \
      (void)cudaStreamSynchronize(st);                                                    \
      return out->status = fail(PAGANI_ERR_CUDA, std::string(#x ": ") + cudaGetErrorString(e)); \
    }                                                                                     \
  } while (0)
  PG_CK(cudaMemcpyAsync(a.ctrl, &h, sizeof(Ctrl), cudaMemcpyHostToDevice, st));
  PG_CK(cudaMemsetAsync(a.probe_acc, 0, sizeof(ProbeAcc) * kProbeBins, st));  // probe bins start at zero
  PG_CK(cudaMemcpyAsync(base + L.prm, &prm, sizeof(prm), cudaMemcpyHostToDevice, st));
  k_uniform_split<<<(int)((s0 + 255) / 256), 256, 0, st>>>(a.pool, d0, log2d, s0);
  PG_CK(cudaGetLastError());
  int launches = 1;
  int64_t d2h = 0;
  for (int guard = 0; guard < h.it_max + 2; ++guard) {
    PG_CK(fk.loop[n](rule, a, Lc.eval_grid, Lc.eval_block, Lc.eval_smem, st));
    ++launches;
    PG_CK(cudaMemcpyAsync(&h, a.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
    PG_CK(cudaStreamSynchronize(st));
    d2h += sizeof(Ctrl);
    if (h.search) {
      for (int probe = 0; probe < 128; ++probe) {
        k_probe<kProbeThreads><<<Lc.probe_grid, kProbeThreads, 0, st>>>(a);
        PG_CK(cudaGetLastError());
        ++launches;
        PG_CK(cudaMemcpyAsync(&h, a.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
        PG_CK(cudaStreamSynchronize(st));
        d2h += sizeof(Ctrl);
        if (!h.search_cont) break;
      }
    }
    k_count<kMgmtThreads, kMgmtItems><<<Lc.count_grid, kMgmtThreads, 0, st>>>(a);
    PG_CK(cudaGetLastError());
    k_split<kMgmtThreads, kMgmtItems><<<Lc.mgmt_grid, kMgmtThreads, 0, st>>>(a);
    PG_CK(cudaGetLastError());
    launches += 2;
    PG_CK(cudaMemcpyAsync(&h, a.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
    PG_CK(cudaStreamSynchronize(st));
    d2h += sizeof(Ctrl);
    if (h.done) break;
  }
#undef PG_CK
  out->estimate = h.estimate;
  out->errorest = h.errorest;
  out->iterations = h.it;
  out->n_regions = h.n_regions_total;
  out->n_active_last = h.s;
  out->finished_volume = nval(h.fin_volume_acc);
  out->active_volume = h.active_volume;
  out->eval_launches = h.it;
  out->kernel_launches = launches;
  out->h2d_bytes = (int64_t)(sizeof(Ctrl) + sizeof(prm));
  out->d2h_bytes = d2h;
  out->n_leaves = -1;
  if (h.watchdog) return out->status = fail(PAGANI_ERR_WATCHDOG, "device-side consistency check failed");
  if (!h.done) return out->status = fail(PAGANI_ERR_WATCHDOG, "loop ended without a result");
  out->status = h.status;
  if (h.status == -6) g_err = "the integrand produced NaN or Inf";
  return out->status;
}

// ======================================================================
// Batched integration: many independent integrals in one graph launch.
// Each instance keeps its own control block (the single-integral Ctrl: the
// same decision code of Algorithms 2 and 3 runs per instance) and a fixed
// slot of slot_cap regions in the pool of its (family, n) group.  Per
// iteration: one Evaluate kernel per group (all instances' pairs), then one
// block per instance reduces, classifies, searches a threshold, compacts and
// splits within its slot.
constexpr int kBatchThreads = 256;
// steps of Algorithm 3 one batch probe launch may take per instance (the
// search itself gives up after 64 probes, so one launch finishes it)
constexpr int kBatchProbeSteps = 64;

__device__ __forceinline__ void batch_slot(const BatchArgs& A, const BatchInst& I, int64_t& base, int64_t& slots,
                                           const BatchGroup*& G) {
  G = &A.groups[I.group];
  slots = (int64_t)G->count * G->slot_cap;
  base = (int64_t)I.local * G->slot_cap;
}

__global__ void __launch_bounds__(kBatchThreads) k_batch_uniform(const BatchArgs A) {
  for (int b = blockIdx.x; b < A.n_inst; b += gridDim.x) {
    const BatchInst& I = A.inst[b];
    const BatchGroup* G;
    int64_t base, slots;
    batch_slot(A, I, base, slots, G);
    const int n = I.n, l0 = I.c.l0, d = 1 << l0;
    const int64_t s0 = I.c.s;
    for (int64_t i = threadIdx.x; i < s0; i += kBatchThreads) {
      int64_t r = i;
      for (int j = n - 1; j >= 0; --j) {
        const int digit = (int)(r & (d - 1));
        r >>= l0;
        G->lower[(size_t)j * slots + base + i] = (double)digit / (double)d;
        G->level[(size_t)j * slots + base + i] = (uint8_t)l0;
      }
    }
  }
}

// Sums, Rel-Err-Classify, termination and the Threshold-Classify trigger of
// every instance (Algorithm 2), one block per instance.
__global__ void __launch_bounds__(kBatchThreads) k_batch_reduce(const BatchArgs A) {
  // staging area of eval_block_finish: 3 * threads + 3 sums and 4 words a warp
  __shared__ __align__(16) unsigned char sh[(3 * kBatchThreads + 3) * sizeof(NSum) + 4 * (kBatchThreads / 32) * 8];
  for (int b = blockIdx.x; b < A.n_inst; b += gridDim.x) {
    BatchInst& I = A.inst[b];
    Ctrl& c = I.c;
    if (c.done) continue;
    const BatchGroup* G;
    int64_t base, slots;
    batch_slot(A, I, base, slots, G);
    const int buf = (c.it - 1) & 1;
    const int64_t s_cur = c.s;  // read once: thread 0 updates c later in this pass
    EvalPartial acc = eval_identity();
    for (int64_t i = threadIdx.x; i < s_cur; i += kBatchThreads) {
      const double v = G->V[base + i], e = G->E[base + i];
      nadd(acc.v, v);
      nadd(acc.e, e);
      acc.emin = fmin(acc.emin, e);
      acc.emax = fmax(acc.emax, e);
      acc.n_rel += relerr_active(v, e, c.tau_cls, c.relerr_filter);
      if (!isfinite(v) || !isfinite(e)) acc.nonfinite = 1;
      int L = 0;
      for (int j = 0; j < I.n; ++j) L += G->level[((size_t)buf * I.n + j) * slots + base + i];
      nadd(acc.vol, pow2_neg(L));
    }
    const EvalPartial tot = eval_block_finish<kBatchThreads>(acc, sh);
    if (threadIdx.x == 0) {
      const int search = finalize_iteration_head(c, nval(tot.v), nval(tot.e), tot.n_rel, tot.emin, tot.emax,
                                                 tot.nonfinite, nullptr, 0, nval(tot.vol));
      if (search) atomicOr(&A.flags[0], 1);
    }
    __syncthreads();
  }
  if (!last_block_arrived(&A.tickets[0])) return;
  if (threadIdx.x == 0) {
    const int any = atomicExch(&A.flags[0], 0);
    A.flags[2] = any;
    set_cond(A.use_graph, A.h_probe, (unsigned)any);
    __threadfence();
  }
}

// One threshold-search probe for every instance still searching (Algorithm 3).
__global__ void __launch_bounds__(kBatchThreads) k_batch_probe(const BatchArgs A) {
  __shared__ unsigned long long sh_lo[kBatchThreads / 32], sh_hi[kBatchThreads / 32];
  __shared__ long long shl[kBatchThreads / 32];
  __shared__ double sh_t;
  __shared__ int sh_cont;
  for (int b = blockIdx.x; b < A.n_inst; b += gridDim.x) {
    BatchInst& I = A.inst[b];
    Ctrl& c = I.c;
    if (c.done || !c.search_cont) continue;
    const BatchGroup* G;
    int64_t base, slots;
    batch_slot(A, I, base, slots, G);
    const int64_t s_cur = c.s;
    const double tau_cls = c.tau_cls;
    const int relerr = c.relerr_filter;
    // the finished candidates' error summed exactly, as the single
    // integral's probe sums it: E / e_b in 128-bit fixed point (e_b = 2^B),
    // so e_abar and every decision of the search are the same bits
    const unsigned long long e_bits = ebits(c.e_b);
    const int B = (e_bits >> 52) ? (int)(e_bits >> 52) - 1023 : -1074 + 63 - __clzll((long long)e_bits);
    if (threadIdx.x == 0) sh_t = c.t;
    __syncthreads();
    // the instance's whole search in this launch: one probe and one step of
    // Algorithm 3 per round (its regions, at most one slot, stay in L2),
    // until the search ends or kBatchProbeSteps steps were taken
    for (int step = 0; step < kBatchProbeSteps; ++step) {
      const double t_cur = sh_t;
      unsigned long long lo = 0ull, hi = 0ull;
      long long na = 0;
      for (int64_t i = threadIdx.x; i < s_cur; i += kBatchThreads) {
        const double e = G->E[base + i];
        if (relerr_active(G->V[base + i], e, tau_cls, relerr) && !(e < t_cur)) {
          ++na;
        } else {
          unsigned long long l, h;
          probe_fixed(ebits(e), e_bits, B, l, h);
          lo += l;
          hi += h + (lo < l ? 1ull : 0ull);
        }
      }
      warp_sum128(lo, hi);
      if ((threadIdx.x & 31) == 0) {
        sh_lo[threadIdx.x >> 5] = lo;
        sh_hi[threadIdx.x >> 5] = hi;
      }
      const long long n = block_sum_ll<kBatchThreads>(na, shl);  // (its barriers publish sh_lo, sh_hi)
      if (threadIdx.x == 0) {
        unsigned long long L = sh_lo[0], H = sh_hi[0];
        for (int w = 1; w < kBatchThreads / 32; ++w) {
          L += sh_lo[w];
          H += sh_hi[w] + (L < sh_lo[w] ? 1ull : 0ull);
        }
        const int cont = threshold_step(c, n, fixed_to_double(L, H, B - kProbeFrac));
        c.search_cont = cont;
        sh_cont = cont;
        sh_t = c.t;
      }
      __syncthreads();
      if (!sh_cont) break;
    }
    if (threadIdx.x == 0 && sh_cont) atomicOr(&A.flags[0], 1);
    __syncthreads();
  }
  if (!last_block_arrived(&A.tickets[1])) return;
  if (threadIdx.x == 0) {
    const int any = atomicExch(&A.flags[0], 0);
    A.flags[2] = any;
    set_cond(A.use_graph, A.h_probe, (unsigned)any);
    __threadfence();
  }
}

// v_f, e_f, the memory check, then Filter + parent update + Split inside the
// instance's slot (Algorithm 2), one block per instance.
__global__ void __launch_bounds__(kBatchThreads) k_batch_split(const BatchArgs A) {
  __shared__ NSum shn[2 * kBatchThreads + 2];
  __shared__ long long shl[kBatchThreads / 32];
  __shared__ int shr[kBatchThreads / 32];
  __shared__ int go_on;
  __shared__ double tau_next;  // the next iteration's tau_cls; pass 2 still classifies with this one's
  for (int b = blockIdx.x; b < A.n_inst; b += gridDim.x) {
    BatchInst& I = A.inst[b];
    Ctrl& c = I.c;
    if (c.done) continue;
    const BatchGroup* G;
    int64_t base, slots;
    batch_slot(A, I, base, slots, G);
    const int n = I.n;
    const int src = (c.it - 1) & 1, dst = src ^ 1;
    const int64_t s_cur = c.s;  // read once: thread 0 rewrites c.s at the end of this pass
    // pass 1: survivors and the finished accumulation (sums of the finished)
    NSum va = {0.0, 0.0}, ea = {0.0, 0.0};
    long long cnt = 0;
    for (int64_t i = threadIdx.x; i < s_cur; i += kBatchThreads) {
      const double v = G->V[base + i], e = G->E[base + i];
      if (final_active(v, e, c)) {
        ++cnt;
      } else {
        nadd(va, v);
        nadd(ea, e);
      }
    }
    NSum t2[2] = {va, ea};
    nsum_block_reduce_staged<kBatchThreads, 2>(t2, shn);
    const NSum tva = t2[0], tea = t2[1];
    const long long n_surv = block_sum_ll<kBatchThreads>(cnt, shl);
    if (threadIdx.x == 0) {
      c.n_surv = n_surv;
      go_on = 0;
      if (2 * n_surv > c.max_regions) {
        c.status = 2;
        c.done = 1;
        c.estimate = c.v + c.vf;
        c.errorest = c.e + c.ef;
      } else {
        const double vf_new = c.vf + nval(tva);
        const double ef_new = c.ef + nval(tea);
        if (n_surv == 0) {  // nothing left to refine: ends as at it_max
          c.status = 1;
          c.done = 1;
          c.estimate = c.v + c.vf;
          c.errorest = c.e + c.ef;
        } else {
          tau_next = survivor_tolerance(c.tau_rel, c.v + c.vf, ef_new, c.v - nval(tva));
          c.vf = vf_new;
          c.ef = ef_new;
          go_on = 1;
        }
      }
    }
    __syncthreads();
    if (go_on) {
      // pass 2: survivors in region order -> children 2q, 2q+1 of the other buffer
      const double* lo_s = G->lower + (size_t)src * n * slots;
      const uint8_t* lv_s = G->level + (size_t)src * n * slots;
      double* lo_d = G->lower + (size_t)dst * n * slots;
      uint8_t* lv_d = G->level + (size_t)dst * n * slots;
      long long run = 0;
      for (int64_t i0 = 0; i0 < s_cur; i0 += kBatchThreads) {
        const int64_t i = i0 + threadIdx.x;
        bool act = false;
        double v = 0.0;
        if (i < s_cur) {
          v = G->V[base + i];
          act = final_active(v, G->E[base + i], c);
        }
        int total;
        const int rank = block_rank<kBatchThreads>(act, shr, &total);
        if (act) {
          const int64_t q = run + rank;
          const int k = G->K[base + i];
          G->Vp[base / 2 + q] = v;
          for (int j = 0; j < n; ++j) {
            const double lo = lo_s[(size_t)j * slots + base + i];
            const int lv = lv_s[(size_t)j * slots + base + i];
            double2 o = make_double2(lo, lo);
            uchar2 ol = make_uchar2((unsigned char)lv, (unsigned char)lv);
            if (j == k) {
              if (lv >= 62) atomicExch(&c.watchdog, 1);
              o.y = lo + pow2_neg(lv + 1);
              ol = make_uchar2((unsigned char)(lv + 1), (unsigned char)(lv + 1));
            }
            *reinterpret_cast<double2*>(lo_d + (size_t)j * slots + base + 2 * q) = o;
            *reinterpret_cast<uchar2*>(lv_d + (size_t)j * slots + base + 2 * q) = ol;
          }
        }
        run += total;
      }
      if (threadIdx.x == 0) {
        c.s = 2 * n_surv;
        c.it += 1;
        c.tau_cls = tau_next;
        atomicOr(&A.flags[1], 1);
      }
    }
    __syncthreads();
  }
  if (!last_block_arrived(&A.tickets[2])) return;
  // live pairs of every instance for the next Evaluate (chunks per thread,
  // chunk sums scanned by warp shuffles)
  {
    __shared__ long long shl[2 * (kBatchThreads / 32)];
    const int nI = A.n_inst;
    const int per = (nI + kBatchThreads - 1) / kBatchThreads;
    const int i0 = threadIdx.x * per, i1 = i0 + per < nI ? i0 + per : nI;
    long long acc = 0;
    for (int i = i0; i < i1; ++i) acc += A.inst[i].c.done ? 0 : A.inst[i].c.s / 2;
    long long total = 0;
    long long run = block_exclusive_scan<kBatchThreads>(acc, shl, &total);
    for (int i = i0; i < i1; ++i) {
      A.pair_prefix[i] = run;
      run += A.inst[i].c.done ? 0 : A.inst[i].c.s / 2;
    }
    if (threadIdx.x == 0) A.pair_prefix[nI] = total;
  }
  if (threadIdx.x == 0) {
    const int any = atomicExch(&A.flags[1], 0);
    A.flags[3] = any;
    set_cond(A.use_graph, A.h_main, (unsigned)any);
    __threadfence();
  }
}

struct BatchWorkspace {
  int dev = -1;
  size_t bytes = 0;
  void* mem = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  std::vector<int64_t> key;   // composition the cached graph was built for
};
static BatchWorkspace g_bws;
static std::map<int, int> g_batch_grid;  // autotuned Evaluate grid per (family, n)

static void release_batch(BatchWorkspace& b) {
  if (b.exec) cudaGraphExecDestroy(b.exec);
  if (b.graph) cudaGraphDestroy(b.graph);
  b.exec = nullptr;
  b.graph = nullptr;
  b.key.clear();
  if (b.mem) cudaFree(b.mem);
  b.mem = nullptr;
  b.bytes = 0;
}

// Bytes of a group's per-instance factor cache (sized for the widest
// element type, the complex factors).
static size_t batch_cache_bytes(const BatchGroup& g) {
  return (size_t)g.count * g.n * kBatchCacheSlots * kCodes * sizeof(double2);
}

static int integrate_batch_locked(int64_t count, const pagani_batch_item* items, int64_t slot_cap_req,
                                  const pagani_options& o, cudaStream_t st, pagani_batch_result* res,
                                  double* ms_out) {
  if (count <= 0 || !items || !res) return fail(PAGANI_ERR_ARGUMENT, "empty batch or null pointer");
  if (count > (1 << 24)) return fail(PAGANI_ERR_ARGUMENT, "batch too large");
  if (o.it_max < 1 || o.it_max > kTraceCap) return fail(PAGANI_ERR_ARGUMENT, "it_max out of range");
  if (o.heuristic_filter < 0 || o.heuristic_filter > 3) return fail(PAGANI_ERR_ARGUMENT, "heuristic_filter must be 0..3");
  if (rule_degree(o.rule_degree) != 9) return fail(PAGANI_ERR_ARGUMENT, "batches use the degree-9 rule");
  int64_t slot_cap = ((slot_cap_req + 1) / 2) * 2;
  // group the instances by (family, n)
  std::map<int, std::vector<int64_t>> by_group;
  for (int64_t i = 0; i < count; ++i) {
    const pagani_batch_item& it = items[i];
    if (it.dim < PAGANI_MIN_DIM || it.dim > PAGANI_MAX_DIM) return fail(PAGANI_ERR_DIM, "item dim must be in [2, 8]");
    if (it.integrand_id < 0 || it.integrand_id >= kNumFamilies) return fail(PAGANI_ERR_INTEGRAND, "unknown integrand_id");
    if (!(it.epsrel > 0.0) || !(it.epsabs >= 0.0)) return fail(PAGANI_ERR_TOLERANCE, "bad item tolerance");
    int rc = check_params(it.integrand_id, it.dim, it.params);
    if (rc) return rc;
    int64_t s0 = 1;
    for (int j = 0; j < it.dim; ++j) s0 *= default_init_div(it.dim);
    if (s0 > slot_cap) return fail(PAGANI_ERR_CAPACITY, "max_regions_per_item below an item's initial split");
    by_group[it.integrand_id * 16 + it.dim].push_back(i);
  }
  std::vector<BatchGroup> groups;
  std::vector<int64_t> order;  // instance position -> item index
  size_t bytes = 0;
  auto align = [](size_t x) { return (x + 255) & ~(size_t)255; };
  bytes += align(sizeof(BatchInst) * count) + align(sizeof(IntegrandParams) * count) + 256 * 4;
  for (auto& kv : by_group) {
    BatchGroup g;
    std::memset(&g, 0, sizeof(g));
    g.family = kv.first / 16;
    g.n = kv.first % 16;
    g.first = (int32_t)order.size();
    g.count = (int32_t)kv.second.size();
    g.slot_cap = slot_cap;
    const size_t slots = (size_t)g.count * slot_cap;
    bytes += align(sizeof(double) * 2 * g.n * slots) + align((size_t)2 * g.n * slots) + 2 * align(8 * slots) +
             align(slots) + align(4 * slots + 8) + align(batch_cache_bytes(g));
    for (int64_t i : kv.second) order.push_back(i);
    groups.push_back(g);
  }
  bytes += align(sizeof(BatchGroup) * groups.size()) + align(sizeof(long long) * (count + 1));
  BatchWorkspace& bw = g_bws;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(PAGANI_ERR_CUDA, cudaGetErrorString(e));
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (bw.dev != dev || bw.bytes < bytes) {
    release_batch(bw);
    e = cudaMalloc(&bw.mem, bytes);
    if (e != cudaSuccess) return fail(PAGANI_ERR_CUDA, std::string("batch workspace: ") + cudaGetErrorString(e));
    bw.bytes = bytes;
    bw.dev = dev;
  }
  // carve the workspace
  unsigned char* p = static_cast<unsigned char*>(bw.mem);
  size_t off = 0;
  auto take = [&](size_t b) {
    unsigned char* q = p + off;
    off += align(b);
    return q;
  };
  BatchArgs a;
  std::memset(&a, 0, sizeof(a));
  a.inst = reinterpret_cast<BatchInst*>(take(sizeof(BatchInst) * count));
  IntegrandParams* prm_d = reinterpret_cast<IntegrandParams*>(take(sizeof(IntegrandParams) * count));
  a.prm = prm_d;
  a.tickets = reinterpret_cast<unsigned int*>(take(256));
  a.flags = reinterpret_cast<int32_t*>(take(256));
  a.pair_prefix = reinterpret_cast<long long*>(take(sizeof(long long) * (count + 1)));
  take(512);
  for (auto& g : groups) {
    const size_t slots = (size_t)g.count * slot_cap;
    g.lower = reinterpret_cast<double*>(take(sizeof(double) * 2 * g.n * slots));
    g.level = take((size_t)2 * g.n * slots);
    g.V = reinterpret_cast<double*>(take(8 * slots));
    g.E = reinterpret_cast<double*>(take(8 * slots));
    g.K = take(slots);
    g.Vp = reinterpret_cast<double*>(take(4 * slots + 8));
    g.fcache = take(batch_cache_bytes(g));
  }
  BatchGroup* groups_d = reinterpret_cast<BatchGroup*>(take(sizeof(BatchGroup) * groups.size()));
  a.groups = groups_d;
  a.n_inst = (int)count;
  // host images of the instance blocks and parameters
  std::vector<BatchInst> hi(count);
  std::vector<IntegrandParams> hp(count);
  for (size_t gi = 0; gi < groups.size(); ++gi) {
    const BatchGroup& g = groups[gi];
    for (int k = 0; k < g.count; ++k) {
      const int64_t pos = g.first + k;
      const pagani_batch_item& it = items[order[pos]];
      BatchInst& I = hi[pos];
      std::memset(&I, 0, sizeof(I));
      I.family = g.family;
      I.n = g.n;
      I.group = (int32_t)gi;
      I.local = k;
      const int d0 = default_init_div(g.n);
      int l0 = 0;
      while ((1 << l0) < d0) ++l0;
      int64_t s0 = 1;
      for (int j = 0; j < g.n; ++j) s0 *= d0;
      Ctrl& c = I.c;
      c.tau_rel = it.epsrel;
      c.tau_cls = it.epsrel;
      c.tau_abs = it.epsabs;
      c.max_regions = slot_cap;
      c.it_max = o.it_max;
      c.relerr_filter = it.relerr_filter ? 1 : 0;
      c.heuristic_filter = trigger_mask(o.heuristic_filter);
      c.s = s0;
      c.it = 1;
      c.status = -100;
      c.l0 = l0;
      hp[pos] = to_params(g.family, g.n, it.params);
    }
  }
#define PG_CK(x)                                                                            \
  do {                                                                                      \
    e = (x);                                                                                \
    if (e != cudaSuccess) return fail(PAGANI_ERR_CUDA, std::string(#x ": ") + cudaGetErrorString(e)); \
  } while (0)
  // live pairs of the first iteration: every instance's s0 / 2
  std::vector<long long> prefix(count + 1, 0);
  for (int64_t i = 0; i < count; ++i) prefix[i + 1] = prefix[i] + hi[i].c.s / 2;
  PG_CK(cudaMemcpyAsync(a.pair_prefix, prefix.data(), sizeof(long long) * (count + 1), cudaMemcpyHostToDevice, st));
  PG_CK(cudaMemcpyAsync(a.inst, hi.data(), sizeof(BatchInst) * count, cudaMemcpyHostToDevice, st));
  PG_CK(cudaMemcpyAsync(prm_d, hp.data(), sizeof(IntegrandParams) * count, cudaMemcpyHostToDevice, st));
  PG_CK(cudaMemcpyAsync(groups_d, groups.data(), sizeof(BatchGroup) * groups.size(), cudaMemcpyHostToDevice, st));
  PG_CK(cudaMemsetAsync(a.tickets, 0, 256, st));
  PG_CK(cudaMemsetAsync(a.flags, 0, 256, st));
  const int inst_grid = (int)std::min<int64_t>(count, (int64_t)sms * 8);
  k_batch_uniform<<<inst_grid, kBatchThreads, 0, st>>>(a);
  PG_CK(cudaGetLastError());
  std::vector<EvalRule> rules(groups.size());
  for (size_t gi = 0; gi < groups.size(); ++gi) {
    const RuleTable* rt = get_rule(groups[gi].n);
    if (!rt) return fail(PAGANI_ERR_CUDA, "rule construction failed");
    rules[gi] = to_eval_rule(*rt);
  }
  // every instance's factor cache, once per call (the parameters are fixed
  // for the whole loop)
  for (size_t gi = 0; gi < groups.size(); ++gi)
    PG_CK(family_kernels(groups[gi].family).batch_fill[groups[gi].n](rules[gi], a, groups[gi], sms * 8, st));
  // autotune each group's Evaluate grid on this batch's first iteration
  std::vector<int> egrid(groups.size());
  cudaEvent_t ev0, ev1;
  PG_CK(cudaEventCreate(&ev0));
  PG_CK(cudaEventCreate(&ev1));
  for (size_t gi = 0; gi < groups.size(); ++gi) {
    const BatchGroup& g = groups[gi];
    const FamilyKernels& fk = family_kernels(g.family);
    const int key = g.family * 16 + g.n;
    auto hit = g_batch_grid.find(key);
    if (hit != g_batch_grid.end()) {
      egrid[gi] = hit->second;
      continue;
    }
    const size_t smem = (size_t)fk.table_bytes_per_thread[g.n] * fk.threads;
    int occ = 0;
    PG_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fk.batch_eval_fn[g.n], fk.threads, smem));
    if (occ < 1) return fail(PAGANI_ERR_CUDA, "batched evaluate kernel does not fit");
    float best = 1e30f;
    int best_grid = sms * occ;
    for (int k = 1; k <= occ; ++k) {
      const int grid = sms * k;
      for (int rep = 0; rep < 2; ++rep) {
        PG_CK(cudaEventRecord(ev0, st));
        PG_CK(fk.batch_eval[g.n](rules[gi], a, g, grid, st));
        PG_CK(cudaEventRecord(ev1, st));
        PG_CK(cudaEventSynchronize(ev1));
        float ms = 0.f;
        PG_CK(cudaEventElapsedTime(&ms, ev0, ev1));
        if (rep == 1 && ms < best) {
          best = ms;
          best_grid = grid;
        }
      }
    }
    g_batch_grid[key] = best_grid;
    egrid[gi] = best_grid;
  }
  PG_CK(cudaEventRecord(ev0, st));
  if (o.use_graph) {
    std::vector<int64_t> key = {count, slot_cap};
    for (size_t gi = 0; gi < groups.size(); ++gi) {
      key.push_back(groups[gi].family * 16 + groups[gi].n);
      key.push_back(groups[gi].count);
      key.push_back(egrid[gi]);
    }
    key.push_back((int64_t)(uintptr_t)bw.mem);
    if (!bw.exec || bw.key != key) {
      if (bw.exec) cudaGraphExecDestroy(bw.exec);
      if (bw.graph) cudaGraphDestroy(bw.graph);
      bw.exec = nullptr;
      bw.graph = nullptr;
      cudaGraph_t gph = nullptr;
      PG_CK(cudaGraphCreate(&gph, 0));
      cudaGraphConditionalHandle hm, hpr;
      cudaGraphNode_t wmain, wprobe, nred, nprobe, nsplit;
      cudaGraph_t body = nullptr, pbody = nullptr;
      PG_CK(cudaGraphConditionalHandleCreate(&hm, gph, 1, cudaGraphCondAssignDefault));
      PG_CK(add_while(&wmain, gph, nullptr, 0, hm, &body));
      PG_CK(cudaGraphConditionalHandleCreate(&hpr, body, 0, 0));
      BatchArgs ga = a;
      ga.use_graph = 1;
      ga.h_main = hm;
      ga.h_probe = hpr;
      std::vector<cudaGraphNode_t> evals(groups.size());
      std::vector<void*> gargs(3 * groups.size());
      std::vector<BatchGroup> gcopy = groups;
      for (size_t gi = 0; gi < groups.size(); ++gi) {
        const FamilyKernels& fk = family_kernels(groups[gi].family);
        gargs[3 * gi] = &rules[gi];
        gargs[3 * gi + 1] = &ga;
        gargs[3 * gi + 2] = &gcopy[gi];
        PG_CK(add_kernel(&evals[gi], body, nullptr, 0, fk.batch_eval_fn[groups[gi].n], egrid[gi], fk.threads,
                         (size_t)fk.table_bytes_per_thread[groups[gi].n] * fk.threads, &gargs[3 * gi]));
      }
      void* margs[1] = {&ga};
      PG_CK(add_kernel(&nred, body, evals.data(), evals.size(), (const void*)&k_batch_reduce, inst_grid,
                       kBatchThreads, 0, margs));
      PG_CK(add_while(&wprobe, body, &nred, 1, hpr, &pbody));
      PG_CK(add_kernel(&nprobe, pbody, nullptr, 0, (const void*)&k_batch_probe, inst_grid, kBatchThreads, 0, margs));
      PG_CK(add_kernel(&nsplit, body, &wprobe, 1, (const void*)&k_batch_split, inst_grid, kBatchThreads, 0, margs));
      PG_CK(cudaGraphInstantiate(&bw.exec, gph, 0));
      bw.graph = gph;
      bw.key = key;
    }
    PG_CK(cudaGraphLaunch(bw.exec, st));
  } else {
    int32_t fl[4];
    for (int guard = 0; guard < o.it_max + 2; ++guard) {
      for (size_t gi = 0; gi < groups.size(); ++gi)
        PG_CK(family_kernels(groups[gi].family).batch_eval[groups[gi].n](rules[gi], a, groups[gi], egrid[gi], st));
      k_batch_reduce<<<inst_grid, kBatchThreads, 0, st>>>(a);
      PG_CK(cudaGetLastError());
      PG_CK(cudaMemcpyAsync(fl, a.flags, sizeof(fl), cudaMemcpyDeviceToHost, st));
      PG_CK(cudaStreamSynchronize(st));
      for (int pr = 0; fl[2] && pr < 128; ++pr) {
        k_batch_probe<<<inst_grid, kBatchThreads, 0, st>>>(a);
        PG_CK(cudaGetLastError());
        PG_CK(cudaMemcpyAsync(fl, a.flags, sizeof(fl), cudaMemcpyDeviceToHost, st));
        PG_CK(cudaStreamSynchronize(st));
      }
      k_batch_split<<<inst_grid, kBatchThreads, 0, st>>>(a);
      PG_CK(cudaGetLastError());
      PG_CK(cudaMemcpyAsync(fl, a.flags, sizeof(fl), cudaMemcpyDeviceToHost, st));
      PG_CK(cudaStreamSynchronize(st));
      if (!fl[3]) break;
    }
  }
  PG_CK(cudaEventRecord(ev1, st));
  PG_CK(cudaMemcpyAsync(hi.data(), a.inst, sizeof(BatchInst) * count, cudaMemcpyDeviceToHost, st));
  PG_CK(cudaStreamSynchronize(st));
  float ms = 0.f;
  PG_CK(cudaEventElapsedTime(&ms, ev0, ev1));
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
#undef PG_CK
  if (ms_out) *ms_out = ms;
  int bad = 0;
  for (int64_t pos = 0; pos < count; ++pos) {
    const Ctrl& c = hi[pos].c;
    pagani_batch_result& r = res[order[pos]];
    r.estimate = c.estimate;
    r.errorest = c.errorest;
    r.status = c.done ? c.status : PAGANI_ERR_WATCHDOG;
    r.iterations = c.it;
    r.n_regions = c.n_regions_total;
    if (c.watchdog) r.status = PAGANI_ERR_WATCHDOG;
    if (!c.done || c.watchdog) bad = 1;
  }
  if (bad) g_err = "some batch items ended without a result (see their status)";
  return 0;
}

}  // namespace pg

// =================================================================== C ABI
using namespace pg;

extern "C" {

void pagani_default_options(pagani_options* o) {
  if (!o) return;
  o->relerr_filter = 1;
  o->heuristic_filter = 1;
  o->init_div = 0;
  o->it_max = 100;
  o->use_graph = 1;
  o->keep_leaves = 0;
  o->rule_degree = 9;
}

int pagani_integrate_box(int dim, int integrand_id, const double* params, const double* lower,
                         const double* upper, double epsrel, double epsabs, int64_t max_regions,
                         const pagani_options* opt, void* cuda_stream, pagani_result* out,
                         pagani_trace_record* trace, int trace_cap) {
  if (!out) return fail(PAGANI_ERR_ARGUMENT, "out is NULL");
  pagani_options o;
  pagani_default_options(&o);
  if (opt) o = *opt;
  std::lock_guard<std::mutex> lk(g_mu);
  try {
    return integrate_locked(dim, integrand_id, params, lower, upper, epsrel, epsabs, max_regions, o,
                            (cudaStream_t)cuda_stream, out, trace, trace_cap);
  } catch (...) {
    return out->status = fail(PAGANI_ERR_CUDA, "internal error");
  }
}

int pagani_integrate_ex(int dim, int integrand_id, const double* params, double epsrel, double epsabs,
                        int64_t max_regions, const pagani_options* opt, void* cuda_stream, pagani_result* out,
                        pagani_trace_record* trace, int trace_cap) {
  return pagani_integrate_box(dim, integrand_id, params, nullptr, nullptr, epsrel, epsabs, max_regions, opt,
                              cuda_stream, out, trace, trace_cap);
}

int pagani_integrate(int dim, int integrand_id, const double* params, double epsrel, double epsabs,
                     int64_t max_regions, pagani_result* out) {
  return pagani_integrate_ex(dim, integrand_id, params, epsrel, epsabs, max_regions, nullptr, nullptr, out,
                             nullptr, 0);
}

int pagani_integrate_noalloc(int dim, int integrand_id, const double* params, double epsrel, double epsabs,
                             int64_t max_regions, void* cuda_stream, pagani_result* out) {
  if (!out) return fail(PAGANI_ERR_ARGUMENT, "out is NULL");
  std::lock_guard<std::mutex> lk(g_mu);
  try {
    return integrate_noalloc_locked(dim, integrand_id, params, epsrel, epsabs, max_regions,
                                    (cudaStream_t)cuda_stream, out);
  } catch (...) {
    return out->status = fail(PAGANI_ERR_CUDA, "internal error");
  }
}

int pagani_integrate_batch(int64_t count, const pagani_batch_item* items, int64_t max_regions_per_item,
                           const pagani_options* opt, void* cuda_stream, pagani_batch_result* results,
                           double* device_ms) {
  pagani_options o;
  pagani_default_options(&o);
  if (opt) o = *opt;
  std::lock_guard<std::mutex> lk(g_mu);
  try {
    cudaStream_t st = cuda_stream ? (cudaStream_t)cuda_stream : nullptr;
    if (!st) {
      int rc = ensure_workspace(4096, 2);
      if (rc) return rc;
      st = g_ws.own_stream;
    }
    return integrate_batch_locked(count, items, max_regions_per_item, o, st, results, device_ms);
  } catch (...) {
    return fail(PAGANI_ERR_CUDA, "internal error");
  }
}

int pagani_workspace_reserve(int64_t max_regions, int dim) {
  if (dim < PAGANI_MIN_DIM || dim > PAGANI_MAX_DIM) return fail(PAGANI_ERR_DIM, "dim must be in [2, 8]");
  if (max_regions < 1) return fail(PAGANI_ERR_ARGUMENT, "max_regions must be positive");
  std::lock_guard<std::mutex> lk(g_mu);
  return ensure_workspace(max_regions, dim);
}

int pagani_workspace_release(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  release_ws(g_ws);
  release_batch(g_bws);
  return 0;
}

int pagani_evaluate(int dim, int integrand_id, const double* params, int64_t m, const double* lower,
                    const double* width, double* V, double* E, int32_t* K, double* diag, void* cuda_stream) {
  return pagani_evaluate_ex(dim, integrand_id, params, 9, m, lower, width, V, E, K, diag, cuda_stream);
}

int pagani_evaluate_ex(int dim, int integrand_id, const double* params, int rule_degree_opt, int64_t m,
                       const double* lower, const double* width, double* V, double* E, int32_t* K, double* diag,
                       void* cuda_stream) {
  if (dim < PAGANI_MIN_DIM || dim > PAGANI_MAX_DIM) return fail(PAGANI_ERR_DIM, "dim must be in [2, 8]");
  const int deg = rule_degree(rule_degree_opt);
  if (deg < 0) return fail(PAGANI_ERR_ARGUMENT, "rule_degree must be 9 (or 0) or 7");
  if (integrand_id < 0 || integrand_id >= kNumFamilies) return fail(PAGANI_ERR_INTEGRAND, "unknown integrand_id");
  if (!params || m < 0) return fail(PAGANI_ERR_ARGUMENT, "bad params or m");
  if (m == 0) return 0;
  if (!lower || !width || !V || !E || !K) return fail(PAGANI_ERR_ARGUMENT, "null device pointer");
  int rc = check_params(integrand_id, dim, params);
  if (rc) return rc;
  std::lock_guard<std::mutex> lk(g_mu);
  const RuleTable* rt = get_rule(dim, deg);
  if (!rt) return fail(PAGANI_ERR_CUDA, "rule construction failed");
  rc = ensure_workspace(4096, dim);
  if (rc) return rc;
  Workspace& w = g_ws;
  cudaStream_t st = cuda_stream ? (cudaStream_t)cuda_stream : w.own_stream;
  const FamilyKernels& fk = family_kernels(integrand_id, deg);
  IntegrandParams prm = to_params(integrand_id, dim, params);
  cudaError_t e = cudaMemcpyAsync(w.prm, &prm, sizeof(prm), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return fail(PAGANI_ERR_CUDA, cudaGetErrorString(e));
  StandaloneArgs a;
  a.lower = lower;
  a.width = width;
  a.V = V;
  a.E = E;
  a.K = K;
  a.diag = diag;
  a.m = m;
  a.prm = w.prm;
  const size_t smem = (size_t)fk.table_bytes_per_thread[dim] * fk.threads;
  const int64_t pairs = (m + 1) / 2;
  int64_t grid = (pairs + fk.threads - 1) / fk.threads;
  if (grid > (int64_t)w.sms * 64) grid = (int64_t)w.sms * 64;
  const EvalRule rule = to_eval_rule(*rt);
  e = diag ? fk.standalone_diag[dim](rule, a, (int)grid, fk.threads, smem, st)
           : fk.standalone[dim](rule, a, (int)grid, fk.threads, smem, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(PAGANI_ERR_CUDA, std::string("evaluate: ") + cudaGetErrorString(e));
  return 0;
}

int pagani_leaves(int dim, int64_t cap, double* lower, uint8_t* level, int64_t* n_out, void* cuda_stream) {
  if (!n_out) return fail(PAGANI_ERR_ARGUMENT, "n_out is NULL");
  std::lock_guard<std::mutex> lk(g_mu);
  Workspace& w = g_ws;
  if (w.last_leaves < 0 || !w.leaves.lower) return fail(PAGANI_ERR_ARGUMENT, "no leaf set kept by the last integration");
  if (dim != w.leaf_n) return fail(PAGANI_ERR_DIM, "dim differs from the kept leaf set");
  *n_out = w.last_leaves;
  if (!lower || !level) return 0;  // size query
  if (cap < w.last_leaves) return fail(PAGANI_ERR_ARGUMENT, "cap below the leaf count");
  cudaStream_t st = cuda_stream ? (cudaStream_t)cuda_stream : w.own_stream;
  const int64_t m = w.last_leaves;
  for (int j = 0; j < dim; ++j) {
    cudaError_t e = cudaMemcpyAsync(lower + (size_t)j * cap, w.leaves.lower + (size_t)j * w.leaves.cap,
                                    sizeof(double) * m, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(level + (size_t)j * cap, w.leaves.level + (size_t)j * w.leaves.cap, m,
                          cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return fail(PAGANI_ERR_CUDA, cudaGetErrorString(e));
  }
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(PAGANI_ERR_CUDA, cudaGetErrorString(e));
  return 0;
}

int pagani_gradient(int dim, int integrand_id, const double* params, int64_t m, const double* lower,
                    const uint8_t* level, double* out, void* cuda_stream) {
  if (dim < PAGANI_MIN_DIM || dim > PAGANI_MAX_DIM) return fail(PAGANI_ERR_DIM, "dim must be in [2, 8]");
  if (integrand_id != kFamProductPeak && integrand_id != kFamGaussian && integrand_id != kFamC0)
    return fail(PAGANI_ERR_INTEGRAND, "gradients exist for the product peak, Gaussian and C0 families");
  if (!params || !out || m < 0) return fail(PAGANI_ERR_ARGUMENT, "bad params, out or m");
  int rc = check_params(integrand_id, dim, params);
  if (rc) return rc;
  std::lock_guard<std::mutex> lk(g_mu);
  const RuleTable* rt = get_rule(dim);
  if (!rt) return fail(PAGANI_ERR_CUDA, "rule construction failed");
  rc = ensure_workspace(4096, dim);
  if (rc) return rc;
  Workspace& w = g_ws;
  const int K = 2 * dim + 1;
  if (m == 0) {
    for (int k = 0; k < K; ++k) out[k] = 0.0;
    return 0;
  }
  if (!lower || !level) return fail(PAGANI_ERR_ARGUMENT, "null device pointer");
  cudaStream_t st = cuda_stream ? (cudaStream_t)cuda_stream : w.own_stream;
  IntegrandParams prm = to_params(integrand_id, dim, params);
  cudaError_t e = cudaMemcpyAsync(w.prm, &prm, sizeof(prm), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return fail(PAGANI_ERR_CUDA, cudaGetErrorString(e));
  // the factor cache, filled for these parameters (the gradient reads the
  // factor values of cached levels from it, as Evaluate does); the launcher
  // then fills the chain-rule terms of the same intervals
  const EvalRule rule = to_eval_rule(*rt);
  {
    LoopArgs la = loop_args(dim, 0, 0, 0);
    int fill_grid = w.sms * 2;
    if (fill_grid > w.max_grid) fill_grid = w.max_grid;
    e = family_kernels(integrand_id).fill[dim](rule, la, fill_grid, 256, 0, st);
    if (e != cudaSuccess) return fail(PAGANI_ERR_CUDA, std::string("factor cache: ") + cudaGetErrorString(e));
  }
  GradArgs a;
  a.lower = lower;
  a.level = level;
  a.m = m;
  a.prm = w.prm;
  a.fcache = static_cast<const double*>(w.fcache);
  a.fcache_levels = kCacheLevels;
  a.terms = w.grad_terms;
  a.part = w.grad_part;
  a.ticket = w.grad_ticket;
  a.out = w.grad_out;
  int64_t grid = (m + kGradThreads - 1) / kGradThreads;
  if (grid > w.max_grid) grid = w.max_grid;
  e = family_kernels(integrand_id).grad[dim](rule, a, (int)grid, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, w.grad_out, sizeof(double) * K, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(PAGANI_ERR_CUDA, std::string("gradient: ") + cudaGetErrorString(e));
  return 0;
}

int pagani_rule_tables(int dim, double* radius, double* weights, int64_t* counts) {
  return pagani_rule_tables_ex(dim, 9, radius, weights, counts);
}

int pagani_rule_tables_ex(int dim, int rule_degree_opt, double* radius, double* weights, int64_t* counts) {
  if (dim < PAGANI_MIN_DIM || dim > PAGANI_MAX_DIM) return fail(PAGANI_ERR_DIM, "dim must be in [2, 8]");
  const int deg = rule_degree(rule_degree_opt);
  if (deg < 0) return fail(PAGANI_ERR_ARGUMENT, "rule_degree must be 9 (or 0) or 7");
  RuleTable t;
  double res = 0.0;
  if (!build_rule(dim, deg, &t, &res)) return fail(PAGANI_ERR_CUDA, "rule construction failed");
  if (radius)
    for (int i = 0; i < 5; ++i) radius[i] = t.radius[i];
  if (weights)
    for (int g = 0; g < kNumGen; ++g)
      for (int k = 0; k < 5; ++k) weights[g * 5 + k] = t.w[g][k];
  if (counts)
    for (int g = 0; g < kNumGen; ++g) counts[g] = t.count[g];
  return t.num_points;
}

int pagani_fp64_peak(double* outv, int n_out, void* cuda_stream) {
  if (!outv || n_out < 1) return fail(PAGANI_ERR_ARGUMENT, "out is NULL");
  std::lock_guard<std::mutex> lk(g_mu);
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const int grid = sms * 4, block = 256;
  double* buf = nullptr;
  cudaError_t e = cudaMalloc(&buf, sizeof(double) * grid * block);
  if (e != cudaSuccess) return fail(PAGANI_ERR_CUDA, cudaGetErrorString(e));
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  auto best_ms = [&](auto launch) {
    launch();  // warm-up
    float best = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
      cudaEventRecord(a, st);
      launch();
      cudaEventRecord(b, st);
      cudaEventSynchronize(b);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, a, b);
      if (ms < best) best = ms;
    }
    return (double)best;
  };
  const int iters = 4096;
  double ms = best_ms([&] { k_fp64_fma<<<grid, block, 0, st>>>(buf, iters, 1.0000001, 1e-9); });
  outv[0] = 2.0 * 8.0 * iters * (double)grid * block / (ms * 1e-3) / 1e12;
  const int citers = 512;
  for (int w = 0; w < 3 && 1 + w < n_out; ++w) {
    ms = best_ms([&] { k_fp64_calls<<<grid, block, 0, st>>>(buf, citers, w); });
    outv[1 + w] = citers * (double)grid * block / (ms * 1e-3) / 1e9;
  }
  e = cudaGetLastError();
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(buf);
  if (e != cudaSuccess) return fail(PAGANI_ERR_CUDA, cudaGetErrorString(e));
  return 0;
}

const char* pagani_last_error(void) { return g_err.c_str(); }

const char* pagani_version(void) { return "pagani-gb300 0.1 (sm_103a, FP64)"; }

}  // extern "C"
