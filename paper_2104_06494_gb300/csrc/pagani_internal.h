// Internal declarations of the GB300 PAGANI engine (not part of the C ABI).
#pragma once
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

namespace pg {

constexpr int kMaxDim = 8;
constexpr int kNumGen = 9;
constexpr int kCodes = 11;  // coordinate codes per axis (see below)

// Noise level of a fourth difference relative to the magnitude sum of its
// five integrand values: at or below it the difference counts as zero in the
// split-axis choice (2^12 unit roundoffs).
constexpr double kDiffNoise = 0x1p-41;

// Per-axis factor cache: the 11 factor values of every dyadic interval
// [k 2^-l, (k+1) 2^-l) of levels l <= kCacheLevels, per axis, slot 2^l - 1 + k.
constexpr int kCacheLevels = 11;
constexpr int kCacheSlots = (1 << (kCacheLevels + 1)) - 1;
// Batches keep a smaller per-instance cache (levels <= kBatchCacheLevels):
// an instance of at most a few ten thousand regions rarely splits an axis
// deeper, and thousands of instances share the device.
constexpr int kBatchCacheLevels = 7;
constexpr int kBatchCacheSlots = (1 << (kBatchCacheLevels + 1)) - 1;

// Generator orbits of the degree-9 rule, in table order.
enum Gen {
  kGenCentre = 0,   // centre
  kGenL1 = 1,       // one axis at sqrt(l1)
  kGenL2 = 2,       // one axis at sqrt(l2)
  kGenL3 = 3,       // one axis at sqrt(l3)
  kGenLp = 4,       // one axis at sqrt(lp) (zero basic weight)
  kGenL1L1 = 5,     // two axes at sqrt(l1)
  kGenL1L2 = 6,     // two axes at sqrt(l1), sqrt(l2), both orders
  kGenL1L1L1 = 7,   // three axes at sqrt(l1)
  kGenL0All = 8     // every axis at sqrt(l0)
};

// Per-axis coordinate codes: the 11 distinct offsets c_j + h_j g a rule point
// can take along one axis.
enum Code {
  kC0 = 0,
  kR1P = 1, kR1M = 2,
  kR2P = 3, kR2M = 4,
  kR3P = 5, kR3M = 6,
  kRpP = 7, kRpM = 8,
  kR0P = 9, kR0M = 10
};

struct RuleTable {
  int n;
  int degree;              // 9: the PAGANI rule; 7: the Genz-Malik variant (error |R7 - R5| = null rule 1)
  int num_points;
  double radius[5];        // sqrt of l1, l2, l3, lp, l0 (on [-1, 1])
  double q;                // fourth-difference weight of the lp and l2 slots, (lp slot / l2 slot)^2 radii:
                           // lp / l2 (degree 9, families with kinks or jumps), 1/7 (degree 7)
  double q_outer;          // weight of the l2 and l1 slots, l2 / l1 (degree 9, smooth families); 0 for degree 7
  double w[kNumGen][5];    // basic rule, null rules 1..4 (unit-volume cube)
  int64_t count[kNumGen];  // orbit sizes
};

bool build_rule(int n, int degree, RuleTable* out, double* max_residual);
std::vector<uint64_t> point_codes(int n);
int num_points(int n);
int64_t orbit_count(int n, int g);

enum Family {
  kFamProductPeak = 0,
  kFamGaussian = 1,
  kFamOscillatory = 2,
  kFamCornerPeak = 3,
  kFamC0 = 4,
  kFamDiscontinuous = 5,
  kFamBoxPower = 6,
  kNumFamilies = 7
};

// Integrand parameters as the kernels read them (device buffer, one per call).
struct IntegrandParams {
  double p0[kMaxDim];   // c (product peak), a (Gaussian, corner peak, C0, oscillatory, discontinuous)
  double p1[kMaxDim];   // w (product peak, Gaussian, C0, discontinuous)
  double u;             // oscillatory phase parameter; box-power exponent
  // integration bounds [a, b] (Algorithm 2): regions live in the unit cube
  // and a point x of it is evaluated at lo + len x; vol = prod len.  The
  // unit cube (lo = 0, len = 1, vol = 1) maps exactly onto itself.
  double lo[kMaxDim];
  double len[kMaxDim];
  double vol;
};

// Neumaier pair used for compensated sums.
struct NSum { double s, c; };

// Device-resident state of one integration; every kernel of the loop reads
// and updates it, the host reads it once at the end.
struct Ctrl {
  // fixed for the call
  double tau_rel, tau_abs;
  int64_t max_regions;
  int32_t it_max, relerr_filter, heuristic_filter, trace_on;
  // iteration state
  int64_t s;                 // regions this iteration
  int32_t it;                // current iteration, 1-based
  int32_t done;              // 1 once the result is final
  int32_t status;            // see pagani.h
  int32_t nonfinite;         // a region produced NaN/Inf
  double v, e, vf, ef;       // Algorithm 2 scalars
  double v_tot_prev;
  double tau_cls;            // Rel-Err-Classify tolerance: the survivors' share
                             // of what tau_rel |v_tot| still allows (tau_rel
                             // until a threshold commit takes more)
  int64_t n_rel;             // rel-err actives this iteration
  double emin, emax;
  int32_t trigger;
  // threshold search (Algorithm 3)
  int32_t search;            // search requested this iteration
  int32_t search_ok, probes, last_dir, dir_changes, search_cont;
  double t, Pmax, e_b;
  // survivors and totals
  int64_t n_surv;
  int64_t n_regions_total;
  double fin_volume;
  NSum fin_volume_acc;
  // result
  double estimate, errorest;
  // last-block tickets
  unsigned int ticket_eval, ticket_probe, ticket_count, ticket_split;
  int32_t watchdog;          // set if a kernel saw an impossible state
  int32_t loop_guard;        // iterations counted by the count kernel
  int32_t total_probes;      // threshold probes (search steps) over the whole call
  int32_t passes;            // probe passes (k_probe launches) this iteration
  int32_t total_passes;      // probe passes over the whole call
  int64_t count_tpb;         // tiles per block of the count kernel (the split locates a tile's block)
  // split kernel: finished E and volume of this iteration as 128-bit fixed
  // point in limbs of 44 bits (value = limb[0] + limb[1] 2^44 + limb[2] 2^88)
  unsigned long long fin_e_fixed[3];
  unsigned long long fin_vol_fixed[3];
  int32_t l0;                // level of the Uniform-Split boxes (log2 of the divisions)
  double active_volume;      // volume of the regions evaluated in the last iteration
  int32_t keep_leaves;       // append finished boxes to the leaf log
  int32_t leaf_overflow;     // the leaf log ran out of room
  int64_t leaf_count;        // boxes in the leaf log before this iteration's
};

// One per-iteration record (mirrors pagani_trace_record in pagani.h).
struct TraceRec {
  int32_t it, trigger, probes, search_ok;
  int64_t s, n_relerr_active, n_survivors;
  double v, e, vf, ef, threshold, direction_changes;
  int32_t probe_passes, reserved;
};

// Per-block partial results written by the evaluate kernel.
struct EvalPartial {
  NSum v, e, vol;
  double emin, emax;
  long long n_rel;
  int nonfinite;
  int pad;
};

struct CountPartial {
  NSum va;                 // V summed over the finished regions of the split kernel's block
  long long n_surv;        // the block's survivors
  long long surv_before;   // survivors of the blocks before it (set by the last block)
};

// Threshold-Classify probes.  One probe pass evaluates the thresholds the
// search can reach from the current threshold t in its next steps: every
// path of kProbeDepth steps (a binary tree: each step moves t halfway to min
// E or to max E), and beyond that the two paths that keep one direction, up
// to kProbeRay steps (runs of same-direction steps are common).  The
// kProbeNodes thresholds, sorted, cut the errors into kProbeBuckets buckets;
// the rel-err finished regions form one more bin.  Each bin sums its errors
// exactly, as integers: E / e_b in fixed point with kProbeFrac fraction bits
// (errors at or above the budget e_b count as e_b, which fails the accuracy
// requirement either way).
constexpr int kProbeDepth = 4;
constexpr int kProbeRay = 8;
constexpr int kProbeTree = (1 << kProbeDepth) - 1;
constexpr int kProbeNodes = kProbeTree + 2 * (kProbeRay - kProbeDepth + 1);
constexpr int kProbeBuckets = kProbeNodes + 1;
constexpr int kProbeBins = kProbeBuckets + 1;
constexpr int kProbeFrac = 88;
constexpr int kProbeThreads = 96;

// One bin of a probe pass, accumulated over all blocks by integer atomics
// (order-independent, so exact and deterministic): the 128-bit fixed-point
// error sum as three limbs, sum = limb[0] + limb[1] 2^44 + limb[2] 2^88
// (each block adds limbs below 2^44, so no carry crosses them and no atomic
// waits for another's result), and the region count.
struct ProbeAcc {
  unsigned long long limb[3], cnt;
};

// Rule data passed by value to the evaluate kernels.
struct EvalRule {
  double radius[5];
  double q;        // fourth-difference weight, lp and l2 slots
  double q_outer;  // fourth-difference weight, l2 and l1 slots (degree 9)
  double noise;  // 64 N(n) u: null values below noise * vol * sum_g |u_kg| M_g count as zero
  double w[kNumGen][5];
  double cnt[kNumGen];  // orbit sizes
  double umax[4];       // max_g |u_kg| (upper bound of the floor's weights)
  double floor_unit[4]; // sum_g |u_kg| cnt_g (the unit-bounded family's floor scale)
  double vround_unit;   // sum_g |w_g| cnt_g (the unit-bounded family's scale of V)
};

// No region error below the rounding level of V itself: 16 u vol sum_g |w_g| M_g.
constexpr double kVRound = 16.0 * 0x1p-53;

// Region pool: SoA, two buffers (ping-pong).  lower[b][j][cap] doubles,
// level[b][j][cap] bytes with width = 2^-level.
struct Pool {
  double* lower;        // 2 * n * cap
  uint8_t* level;       // 2 * n * cap
  double* V;            // cap
  double* E;            // cap
  uint8_t* K;           // cap
  uint8_t* act;         // cap: Rel-Err-Classify of the iteration (written by Evaluate), then the
                        // final classification (the count kernel clears threshold-finished ones)
  double* Vp;           // cap / 2 + 1
  int* tile_count;         // (n_tiles + 1) * kTileWarps: survivors per warp slice of a tile
  long long* tile_offset;  // n_tiles + 1
  int64_t cap;
  int n;
};

// Leaf log: the boxes classified finished, appended per iteration, and at
// the end every box of the last iteration (SoA [n][cap]).
struct LeafLog {
  double* lower;
  uint8_t* level;
  int64_t cap;
};

// Arguments of the loop kernels (by value).
struct LoopArgs {
  Pool pool;
  Ctrl* ctrl;
  const IntegrandParams* prm;
  EvalPartial* eval_part;
  ProbeAcc* probe_acc;     // kProbeBins bins, zero between probe passes
  CountPartial* count_part;
  TraceRec* trace;
  int trace_cap;
  int use_graph;
  cudaGraphConditionalHandle h_main, h_probe;
  void* fcache;          // per-axis factor cache (element type of the family), or null
  int fcache_levels;     // deepest cached level
  LeafLog leaves;        // leaf log (null pointers: none)
  // packed rule points of dimension pool.n (see point_codes), generator g at
  // [gen_off[g], gen_off[g + 1]); null: Evaluate always runs thread per pair
  const uint64_t* codes;
  int gen_off[kNumGen + 1];
};

// Evaluate's three forms, by the number of regions s of the iteration:
//  * one warp per sibling pair while the pairs fit in kCoopPasses passes of
//    all the launch's warps;
//  * one thread per region (sibling lanes exchange values for the two-level
//    estimate) while the regions fit in kRegionPasses passes of its threads;
//  * one thread per sibling pair (the shared factor table) beyond.
// A warp alone on a scheduler runs its dependent FP64 chains at about 64
// cycles per step, so while few warps exist, halving each warp's chain
// (a region instead of a pair) shortens the launch.
constexpr int kCoopPasses = 1;
constexpr int kRegionPasses = 2;

// Arguments of the gradient kernel.
struct GradArgs {
  const double* lower;     // [n][m]
  const uint8_t* level;    // [n][m]
  int64_t m;
  const IntegrandParams* prm;
  const double* fcache;    // per-axis factor cache filled for prm (levels <= fcache_levels), or null
  int fcache_levels;
  double* terms;           // [n][kCacheSlots][kGradTerms] chain-rule terms, filled by the launcher
  double* part;            // per block: 2n + 1 Neumaier pairs (value, gradient)
  unsigned int* ticket;
  double* out;             // 2n + 1 totals (value first)
};
typedef cudaError_t (*GradLauncher)(const EvalRule&, const GradArgs&, int grid, cudaStream_t);
constexpr int kGradThreads = 64;  // gradient kernel: one thread per box
constexpr int kGradTerms = 10;    // chain-rule terms per axis interval (centre + 4 radii, 2 parameters)

// Arguments of the standalone evaluate entry point.
struct StandaloneArgs {
  const double* lower;   // n x m SoA
  const double* width;   // n x m SoA
  double* V;
  double* E;
  int32_t* K;
  double* diag;          // (8 + n) x m SoA or null
  int64_t m;
  const IntegrandParams* prm;
};

// ------------------------------------------------------------------ batch
// One instance of a batch: its loop state (the single-integral control
// block, reused) and where its regions live.  Instances of one (family, n)
// group share a pool; instance k of the group owns regions
// [k * slot_cap, (k + 1) * slot_cap).
struct BatchInst {
  Ctrl c;
  int32_t family, n, group, local;
};

struct BatchGroup {
  int32_t family, n, first, count;   // instances [first, first + count)
  int64_t slot_cap;
  double* lower;    // [2][n][count * slot_cap]
  uint8_t* level;   // [2][n][count * slot_cap]
  double* V;
  double* E;
  uint8_t* K;
  double* Vp;       // [count * slot_cap / 2]
  void* fcache;     // [count][n][kBatchCacheSlots][kCodes] factor values (family element type)
};

struct BatchArgs {
  BatchInst* inst;
  const IntegrandParams* prm;   // per instance
  const BatchGroup* groups;     // device copy
  int n_inst;
  unsigned int* tickets;        // [0] reduce, [1] probe, [2] split
  int32_t* flags;               // [0] any searching, [1] any running
  // exclusive prefix over the instances (group order) of their live pairs
  // (s / 2, or 0 once done); [n_inst] is the total.  Evaluate visits only these.
  long long* pair_prefix;
  int use_graph;
  cudaGraphConditionalHandle h_main, h_probe;
};

// Launchers implemented per family (eval_<family>.cu).
typedef cudaError_t (*LoopEvalLauncher)(const EvalRule&, const LoopArgs&, int grid, int block, size_t smem,
                                        cudaStream_t);
typedef cudaError_t (*StandaloneLauncher)(const EvalRule&, const StandaloneArgs&, int grid, int block,
                                          size_t smem, cudaStream_t);

struct FamilyKernels {
  LoopEvalLauncher loop[kMaxDim + 1];
  LoopEvalLauncher fill[kMaxDim + 1];      // factor-cache fill, one level per iteration
  const void* fill_fn[kMaxDim + 1];
  StandaloneLauncher standalone[kMaxDim + 1];
  StandaloneLauncher standalone_diag[kMaxDim + 1];
  const void* loop_fn[kMaxDim + 1];        // kernel symbols (for occupancy queries / graph nodes)
  GradLauncher grad[kMaxDim + 1];          // gradient over a box list (positive product families)
  cudaError_t (*batch_eval[kMaxDim + 1])(const EvalRule&, const BatchArgs&, const BatchGroup&, int grid,
                                         cudaStream_t);
  cudaError_t (*batch_fill[kMaxDim + 1])(const EvalRule&, const BatchArgs&, const BatchGroup&, int grid,
                                         cudaStream_t);
  const void* batch_eval_fn[kMaxDim + 1];
  int threads;                             // block size
  int table_bytes_per_thread[kMaxDim + 1];
};

const FamilyKernels& kernels_product_peak();
const FamilyKernels& kernels_gaussian();
const FamilyKernels& kernels_oscillatory();
const FamilyKernels& kernels_corner_peak();
const FamilyKernels& kernels_c0();
const FamilyKernels& kernels_discontinuous();
const FamilyKernels& kernels_box_power();
// the Genz-Malik degree-7 variants (loop, cache fill, standalone)
const FamilyKernels& kernels_product_peak_gm7();
const FamilyKernels& kernels_gaussian_gm7();
const FamilyKernels& kernels_oscillatory_gm7();
const FamilyKernels& kernels_corner_peak_gm7();
const FamilyKernels& kernels_c0_gm7();
const FamilyKernels& kernels_discontinuous_gm7();
const FamilyKernels& kernels_box_power_gm7();

constexpr int kSplitThreads = 256;
constexpr int kItemsPerThread = 8;
constexpr int kTile = kSplitThreads * kItemsPerThread;  // regions per compaction tile
constexpr int kTileWarps = 8;  // warp slices per tile in the survivor count (256 regions each)
constexpr int kReduceThreads = 256;

}  // namespace pg
