/*
 * Plain CPU oracle of the PAGANI adaptive integration loop.
 *
 * ORACLE / TEST INFRASTRUCTURE ONLY.  This file shares no code with the CUDA
 * path and is never linked into the product library.  Only tests/, the smoke
 * check and the CPU-baseline leg of bench.py load it (through oracle/capi.py).
 *
 * It follows the paper's "PAGANI Algorithm" (Sec. 3.1, Algorithm 2) and
 * "Threshold Classification" (Sec. 3.5.3, Algorithm 3) step by step in the
 * paper's order and notation: Uniform-Split, then per iteration Evaluate,
 * Two-Level-Error, Rel-Err-Classify, Sum(V), Sum(E), the termination test,
 * Threshold-Classify, the finished accumulations v_f and e_f, Filter, the
 * parent update and Split.  Everything is double precision, single threaded,
 * summed in region-index order, and compiled with -ffp-contract=off so the
 * results are the same on x86-64 and aarch64.
 *
 * Readings of passages the paper leaves open:
 *  - Evaluate (Sec. 3.2): the rule, its null rules and the error formula come
 *    in as tables from oracle/rule.py.  The four null values N_1..N_4
 *    (degrees 7, 5, 3, 1) are differences between the basic rule and
 *    embedded lower-degree rules; on a box where f is resolved they fall
 *    off geometrically with the degree, by a ratio r per two degrees, and
 *    the degree-9 rule's own error is about r N_1.  So:
 *      r = max(N_1/N_2, N_2/N_3, N_3/N_4)  (x/0 = inf for x > 0, 0 for x = 0);
 *      r >= 1 (no decay: f not resolved): err = 10 max(N_1, N_2, N_3), the
 *        largest difference of the rules of degree >= 3;
 *      r <  1: err = 10 r max(N_1, r N_2), where r N_2 stands in for a
 *        degree-7 value that cancelled by accident (N_1 far below the
 *        geometric trend of the others).
 *    The factor 10 is a safety margin: on degree-10 terms the rule's error
 *    is 0.3 to 1.2 times N_1, so err overstates a resolved box's error by
 *    about 10 to 30.  A null value N_k no larger than
 *    64 N(n) u vol sum_g |u_kg| M_g (u the unit roundoff, M_g the magnitude
 *    of orbit sum S_g: |S_g| for the positive families, the orbit size for
 *    the oscillatory one, |f| <= 1) is at the rounding level of its sum and
 *    counts as zero.  The error is never below the rounding level of V
 *    itself, 16 u vol sum_g |w_g| M_g: no rule sum is more accurate than a
 *    few unit roundoffs of its absolute sum.
 *  - Split axis (Sec. 2.2, Sec. 3.2): fourth divided difference per axis,
 *    D_j = |(f(c+a h_j e_j) + f(c-a h_j e_j) - 2 f(c))
 *           - q (f(c+b h_j e_j) + f(c-b h_j e_j) - 2 f(c))|, q = a^2/b^2,
 *    with radii a < b of the rule's one-axis orbits (they come in with the
 *    rule, per family, from oracle/capi.py): the inner and the outer
 *    radius a = sqrt(l2), b = sqrt(l1) for smooth integrands, as Genz and
 *    Malik's rule does with sqrt(9/70), sqrt(9/10) (the degree-7 variant's
 *    radii); the two inner radii a = sqrt(lp), b = sqrt(l2) for the C0 and
 *    discontinuous families, whose kinks and jumps, once a difference
 *    reaching out to sqrt(l1) has bisected a box across them, can sit in
 *    the outer margin of a child beyond every rule point, where no error
 *    estimate sees them;
 *    a D_j no larger than 2^12 u M_j (M_j the same sum over |f|) is rounding
 *    noise and counts as zero; K = smallest j with D_j >= (1 - 1e-10) max D;
 *    if every D_j counts as zero, the widest axis (smallest j among equals).
 *  - Two-level error (Sec. 2.1, Sec. 3.2): for siblings L, R of parent P,
 *    delta = |V_L + V_R - V_P| / 4, S = E_L + E_R; if S > 0 each child's error
 *    becomes E (1 + 2 delta / S) + delta, else E + delta.
 *  - Uniform-Split (Sec. 3.1): d = largest power of two >= 2 with d^n <= 4096.
 *  - Children of survivor p are stored at 2p (lower half) and 2p+1 (upper
 *    half), so the parent of region i is i/2 and its sibling i^1.
 *  - Threshold-Classify trigger (Sec. 3.5.2): (a) from the second iteration
 *    on, |v_tot - v_tot_prev| <= tau_rel |v_tot|; (b) 2 (number of rel-err
 *    actives) > max_regions.
 *  - Threshold search (Sec. 3.5.3): the error budget is the part of the
 *    tolerance that finished regions may still take, e_b = tau_rel |v_tot| -
 *    e_f: finished error above it makes convergence impossible, which the
 *    search avoids by its choice of threshold (accuracy requirement
 *    e_abar <= P_max e_b, P_max <= 0.95); no search when e_b <= 0.  e_b is
 *    rounded down to a power of two: once most of the tolerance is spent it
 *    is a difference of nearly equal sums, whose low bits are rounding.
 *  - Sums of Algorithm 2/3 that are small differences of large sums are
 *    formed directly: e_abar (= e_it - sum A.E) as the sum of E over the
 *    finished candidates, v - sum V.A and e - sum E.A over the finished
 *    regions.  Equal in exact arithmetic; the direct sums carry the
 *    rounding of the finished part only.
 *    The first threshold is the mean error and the range [min, max] of the
 *    errors, rounded to powers of two (the mean down, min down, max up):
 *    errors carry the rounding of the null-rule and two-level differences
 *    they come from, and rounded inputs let two implementations of the same
 *    arithmetic probe the same thresholds.
 *    Candidate finished set = rel-err finished plus {E_i < t}; too few
 *    finished -> t += (max - t)/2; too much error -> t -= (t - min)/2; every
 *    change of direction adds 0.10 to P_max (cap 0.95); give up after 10
 *    direction changes or 64 probes.
 *  - Rel-Err-Classify after a threshold commit (Sec. 3.5.1, Sec. 3.5.2): the
 *    Lemma bounds the rel-err finished regions' error by tau times their
 *    integral only while no other finished error has used up the tolerance.
 *    Regions are therefore finished iff E_i <= tau_cls |V_i|, where tau_cls =
 *    min(tau_rel, (tau_rel |v_tot| - e_f) / |sum of the survivors' V|) is the
 *    survivors' share of what the tolerance still allows, set after each
 *    iteration's finished accumulation (tau_rel at the start).  Without
 *    threshold commits tau_cls = tau_rel for a same-sign integrand.  A share
 *    below tau_rel is rounded down to a power of two: once most of the
 *    tolerance is spent, the allowance is a difference of nearly equal sums
 *    whose rounding would otherwise move the tolerance itself.
 *  - Memory exhaustion (Sec. 3.5.2): if 2 (survivors) > max_regions after
 *    the threshold step, return the latest estimates with status 2.
 *  - When no region stays active (possible only if rel-err filtering runs on
 *    a sign-changing integrand), later iterations could not change v + v_f or
 *    e + e_f, so the loop ends at once with the it_max status 1.
 *  Parity unpinned: the error formula's constants and noise floors and the
 *  two-level formula are readings with no published values to pin them to;
 *  they are checked through estimates staying within their error estimates
 *  of closed forms, and through error estimates not overstating the true
 *  error by orders of magnitude on smooth integrands.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_PI 3.14159265358979323846

enum {
  FAM_PRODUCT_PEAK = 0,
  FAM_GAUSSIAN = 1,
  FAM_OSCILLATORY = 2,
  FAM_CORNER_PEAK = 3,
  FAM_C0 = 4,
  FAM_DISCONTINUOUS = 5,
  FAM_BOX_POWER = 6,
  FAM_MONOMIAL = 100 /* test-only: prod_j x_j^(p_j), integer p_j */
};

typedef struct {
  int n;              /* dimension */
  int G;              /* number of generators */
  const double *gen;  /* G x n generator magnitudes on [-1,1]^n, row-major */
  const double *wts;  /* G x 5: basic rule, then null rules u_1..u_4 */
  double a, b, q;     /* fourth-difference radii: inner a, outer b; q = a^2/b^2 */
  const int64_t *count; /* G orbit sizes */
  int error_kind;     /* 0: the four-null-rule error formula (degree-9 rule);
                         1: |R7 - R5|, the Genz-Malik degree-7 rule's difference
                         with its embedded degree-5 rule (null rule 1 = w7 - w5) */
} oracle_rule;

typedef struct {
  int relerr_filter;     /* Sec. 3.5.1: 0 turns rel-err classification off */
  int heuristic_filter;  /* Sec. 3.5.2 triggers of Threshold-Classify: 1 both,
                            2 memory only, 3 unchanged digits only, 0 off */
  int init_div;          /* 0 = default Uniform-Split divisions */
  int it_max;
  const double *lower;   /* integration bounds a[n], b[n] of Algorithm 2;  */
  const double *upper;   /* both NULL: the unit cube                        */
} oracle_options;

typedef struct {
  double estimate, errorest;
  int status;            /* 0 converged, 1 it_max (or no region left
                            active), 2 memory exhausted, <0 error */
  int iterations;
  int64_t n_regions;     /* sum over iterations of regions evaluated */
  int64_t n_active_last; /* regions evaluated in the last iteration */
} oracle_result;

typedef struct {
  int32_t it, trigger, probes, search_ok;
  int64_t s, n_relerr_active, n_survivors;
  double v, e, vf, ef, threshold, direction_changes;
} oracle_trace;

/* ------------------------------------------------------------ integrands -- */
static double integrand(int fam, int n, const double *p, const double *x) {
  double s = 0.0, r = 1.0;
  int j;
  switch (fam) {
  case FAM_PRODUCT_PEAK: /* prod_j 1/(c_j^-2 + (x_j - w_j)^2); p = c[n], w[n] */
    for (j = 0; j < n; ++j) {
      double t = x[j] - p[n + j];
      r *= 1.0 / (pow(p[j], -2.0) + t * t);
    }
    return r;
  case FAM_GAUSSIAN: /* exp(-sum_j a_j^2 (x_j - w_j)^2); p = a[n], w[n] */
    for (j = 0; j < n; ++j) {
      double t = x[j] - p[n + j];
      s += p[j] * p[j] * t * t;
    }
    return exp(-s);
  case FAM_OSCILLATORY: /* cos(2 pi u + sum_j a_j x_j); p = u, a[n] */
    s = 2.0 * OR_PI * p[0];
    for (j = 0; j < n; ++j) s += p[1 + j] * x[j];
    return cos(s);
  case FAM_CORNER_PEAK: /* (1 + sum_j a_j x_j)^-(n+1); p = a[n] */
    s = 1.0;
    for (j = 0; j < n; ++j) s += p[j] * x[j];
    return pow(s, -(double)(n + 1));
  case FAM_C0: /* exp(-sum_j a_j |x_j - w_j|); p = a[n], w[n] */
    for (j = 0; j < n; ++j) s += p[j] * fabs(x[j] - p[n + j]);
    return exp(-s);
  case FAM_DISCONTINUOUS: /* exp(sum_j a_j x_j) if every x_j < w_j, else 0; p = a[n], w[n] */
    for (j = 0; j < n; ++j) {
      if (!(x[j] < p[n + j])) return 0.0;
      s += p[j] * x[j];
    }
    return exp(s);
  case FAM_BOX_POWER: /* (sum_j x_j^2)^q; p = q */
    for (j = 0; j < n; ++j) s += x[j] * x[j];
    return pow(s, p[0]);
  case FAM_MONOMIAL:
    for (j = 0; j < n; ++j) {
      int e, k = (int)p[j];
      for (e = 0; e < k; ++e) r *= x[j];
    }
    return r;
  }
  return NAN;
}

/* ------------------------------------------------------ orbit enumeration -- */
/* next lexicographic permutation of v[0..n) (ascending order); 0 at the end */
static int next_perm(double *v, int n) {
  int i = n - 2, k;
  while (i >= 0 && !(v[i] < v[i + 1])) --i;
  if (i < 0) return 0;
  k = n - 1;
  while (!(v[i] < v[k])) --k;
  { double t = v[i]; v[i] = v[k]; v[k] = t; }
  for (int lo = i + 1, hi = n - 1; lo < hi; ++lo, --hi) {
    double t = v[lo]; v[lo] = v[hi]; v[hi] = t;
  }
  return 1;
}

static int cmp_double(const void *a, const void *b) {
  double x = *(const double *)a, y = *(const double *)b;
  return (x > y) - (x < y);
}

/* Sum of f over the orbit of one generator (all distinct coordinate
 * permutations, all sign changes of the non-zero coordinates) on the box with
 * centre c and half-widths h.  Also returns the sum of |f| and the count. */
static double orbit_sum(int fam, int n, const double *p, const double *genrow,
                        const double *c, const double *h, double *abs_sum,
                        int64_t *count) {
  double v[16], x[16], s = 0.0, sa = 0.0;
  int64_t cnt = 0;
  memcpy(v, genrow, sizeof(double) * n);
  qsort(v, n, sizeof(double), cmp_double);
  do {
    int nzi[16], nz = 0;
    for (int j = 0; j < n; ++j)
      if (v[j] != 0.0) nzi[nz++] = j;
    for (int mask = 0; mask < (1 << nz); ++mask) {
      for (int j = 0; j < n; ++j) x[j] = c[j];
      for (int t = 0; t < nz; ++t) {
        int j = nzi[t];
        double g = (mask >> t & 1) ? -v[j] : v[j];
        x[j] = c[j] + h[j] * g;
      }
      double f = integrand(fam, n, p, x);
      s += f;
      sa += fabs(f);
      ++cnt;
    }
  } while (next_perm(v, n));
  *abs_sum = sa;
  *count = cnt;
  return s;
}

/* --------------------------------------------------------------- Evaluate -- */
static double ratio_or(double x, double y) {
  if (y > 0.0) return x / y;
  return x > 0.0 ? INFINITY : 0.0;
}

/* The region error from the four null-rule values (reading given above). */
static double null_rule_error(const double N[4]) {
  double r = fmax(fmax(ratio_or(N[0], N[1]), ratio_or(N[1], N[2])), ratio_or(N[2], N[3]));
  if (r >= 1.0) return 10.0 * fmax(fmax(N[0], N[1]), N[2]);
  return 10.0 * r * fmax(N[0], r * N[1]);
}

/* Evaluate one region [lower, lower + width]: integral V, null-rule error E,
 * split axis K.  diag (if not NULL) receives N_1..N_4, the four sums
 * vol * sum_g |u_kg| * sum_orbit |f| (rounding scale of N_k), the rounding
 * scale of V, then D_0..D_{n-1} and the rounding scales of the D_j. */
static void evaluate_region(const oracle_rule *R, int fam, const double *p,
                            const double *lower, const double *width, double *V,
                            double *E, int *K, double *diag) {
  int n = R->n;
  double c[16], h[16], vol = 1.0;
  double Sg[32], Ag[32];
  for (int j = 0; j < n; ++j) {
    h[j] = 0.5 * width[j];
    c[j] = lower[j] + h[j];
    vol *= width[j];
  }
  for (int g = 0; g < R->G; ++g) {
    int64_t cnt;
    Sg[g] = orbit_sum(fam, n, p, R->gen + (size_t)g * n, c, h, &Ag[g], &cnt);
  }
  double basic = 0.0, basic_abs = 0.0, basic_mag = 0.0, N[4], Nabs[4], Nfloor[4], Nused[4];
  int64_t npts = 0;
  for (int g = 0; g < R->G; ++g) {
    basic += R->wts[g * 5] * Sg[g];
    basic_abs += fabs(R->wts[g * 5]) * Ag[g];
    basic_mag += fabs(R->wts[g * 5]) * (fam == FAM_OSCILLATORY ? (double)R->count[g] : fabs(Sg[g]));
  }
  for (int g = 0; g < R->G; ++g) npts += R->count ? R->count[g] : 0;
  for (int k = 0; k < 4; ++k) {
    double s = 0.0, sa = 0.0, sc = 0.0;
    for (int g = 0; g < R->G; ++g) {
      s += R->wts[g * 5 + 1 + k] * Sg[g];
      sa += fabs(R->wts[g * 5 + 1 + k]) * Ag[g];
      /* magnitude of the orbit sum: |S_g| = sum |f| for the positive
       * families; |f| <= 1 bounds it by the orbit size for the oscillatory
       * one, whose values carry absolute rounding errors */
      double mag = fam == FAM_OSCILLATORY ? (double)R->count[g] : fabs(Sg[g]);
      sc += fabs(R->wts[g * 5 + 1 + k]) * mag;
    }
    N[k] = vol * fabs(s);
    Nabs[k] = vol * sa;
    /* a null value at the rounding level of its own sum carries no
     * information and counts as zero */
    Nfloor[k] = 64.0 * (double)npts * 0x1p-53 * (vol * sc);
    Nused[k] = N[k] <= Nfloor[k] ? 0.0 : N[k];
  }
  *V = vol * basic;
  *E = R->error_kind == 1 ? Nused[0] : null_rule_error(Nused);
  /* no error below the rounding level of V itself */
  double Vround = 16.0 * 0x1p-53 * (vol * basic_mag);
  if (*E < Vround) *E = Vround;

  /* split axis from fourth divided differences */
  double x[16], D[16], Dabs[16], Dused[16], f0, Dmax = 0.0;
  for (int j = 0; j < n; ++j) x[j] = c[j];
  f0 = integrand(fam, n, p, x);
  for (int j = 0; j < n; ++j) {
    double fa_p, fa_m, fb_p, fb_m;
    x[j] = c[j] + h[j] * R->a; fa_p = integrand(fam, n, p, x);
    x[j] = c[j] - h[j] * R->a; fa_m = integrand(fam, n, p, x);
    x[j] = c[j] + h[j] * R->b; fb_p = integrand(fam, n, p, x);
    x[j] = c[j] - h[j] * R->b; fb_m = integrand(fam, n, p, x);
    x[j] = c[j];
    D[j] = fabs((fa_p + fa_m - 2.0 * f0) - R->q * (fb_p + fb_m - 2.0 * f0));
    Dabs[j] = fabs(fa_p) + fabs(fa_m) + 2.0 * fabs(f0) +
              R->q * (fabs(fb_p) + fabs(fb_m) + 2.0 * fabs(f0));
    /* a difference within rounding noise of zero (2^12 unit roundoffs of
     * the magnitude of its five values) tells nothing about the axis */
    Dused[j] = D[j] <= 4096.0 * 0x1p-53 * Dabs[j] ? 0.0 : D[j];
    if (Dused[j] > Dmax) Dmax = Dused[j];
  }
  /* the largest difference, near-ties to the lowest axis; every difference
   * at its noise floor: the widest axis, ties to the lowest */
  int k = 0;
  if (Dmax > 0.0) {
    while (!(Dused[k] >= (1.0 - 1e-10) * Dmax)) ++k;
  } else {
    for (int j = 1; j < n; ++j)
      if (width[j] > width[k]) k = j;
  }
  *K = k;
  if (diag) {
    for (int t = 0; t < 4; ++t) diag[t] = N[t];
    for (int t = 0; t < 4; ++t) diag[4 + t] = Nabs[t];
    diag[8] = vol * basic_abs;
    for (int j = 0; j < n; ++j) diag[9 + j] = D[j];
    for (int j = 0; j < n; ++j) diag[9 + n + j] = Dabs[j];
    for (int t = 0; t < 4; ++t) diag[9 + 2 * n + t] = Nfloor[t];
  }
}

/* Exported: evaluate m regions (row-major lower/width, m x n). */
int oracle_evaluate(const oracle_rule *R, int fam, const double *params,
                    int64_t m, const double *lower, const double *width,
                    double *V, double *E, int32_t *K, double *diag) {
  for (int64_t i = 0; i < m; ++i) {
    int k;
    evaluate_region(R, fam, params, lower + i * R->n, width + i * R->n, &V[i],
                    &E[i], &k, diag ? diag + i * (13 + 2 * R->n) : NULL);
    K[i] = k;
  }
  return 0;
}

/* ----------------------------------------------------- Neumaier summation -- */
typedef struct { double s, c; } nsum;
static void nadd(nsum *a, double x) {
  double t = a->s + x;
  if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
  else a->c += (x - t) + a->s;
  a->s = t;
}
static double nval(const nsum *a) { return a->s + a->c; }

/* ---------------------------------------------------- Two-Level-Error ---- */
static void two_level_error(int64_t s, const double *V, double *E,
                            const double *Vp) {
  for (int64_t p = 0; p < s / 2; ++p) {
    int64_t L = 2 * p, Rr = 2 * p + 1;
    double delta = fabs(V[L] + V[Rr] - Vp[p]) / 4.0;
    double S = E[L] + E[Rr];
    if (S > 0.0) {
      double cc = 1.0 + 2.0 * delta / S;
      E[L] = E[L] * cc + delta;
      E[Rr] = E[Rr] * cc + delta;
    } else {
      E[L] += delta;
      E[Rr] += delta;
    }
  }
}

/* --------------------------------------------------- Rel-Err-Classify ---- */
static void rel_err_classify(int64_t s, const double *V, const double *E,
                             double tau_rel, int enabled, uint8_t *A) {
  for (int64_t i = 0; i < s; ++i)
    A[i] = enabled ? !(E[i] <= tau_rel * fabs(V[i])) : 1;
}

/* ------------------------------------------------- Threshold-Classify ---- */
/* Returns 1 and updates A when a threshold meets the memory and accuracy
 * requirements; otherwise leaves A unchanged (unsuccessful filtering).
 * v_tot = v + v_f, e_f the error finished in earlier iterations, e_it and
 * s_it this iteration's error sum and region count. */
static int threshold_classify(uint8_t *A, const double *E, double v_tot,
                              double e_f, double e_it, int64_t s_it,
                              double tau_rel, int *probes_out, double *t_out,
                              int *dirchg_out) {
  double Pmax = 0.25;
  double mn = INFINITY, mx = -INFINITY;
  for (int64_t i = 0; i < s_it; ++i) {
    if (E[i] < mn) mn = E[i];
    if (E[i] > mx) mx = E[i];
  }
  /* the search range [min, max] rounded outward to powers of two */
  if (mn > 0.0) { int ex; frexp(mn, &ex); mn = ldexp(0.5, ex); }
  if (mx > 0.0) { int ex; double m = frexp(mx, &ex); mx = m == 0.5 ? mx : ldexp(1.0, ex); }
  /* error budget: what the finished regions may still add before the
     tolerance tau_rel |v_tot| is out of reach, rounded down to a power of
     two (a difference of nearly equal sums once most of the tolerance is
     spent: its low bits are the rounding of e_f) */
  double e_b = fabs(v_tot) * tau_rel - e_f;
  if (e_b > 0.0) {
    int ex;
    frexp(e_b, &ex);
    e_b = ldexp(0.5, ex);
  }
  /* start: the mean error, rounded down to a power of two */
  double t = e_it / (double)s_it;
  if (t > 0.0) { int ex; frexp(t, &ex); t = ldexp(0.5, ex); }
  int probes = 0, last_dir = 0, changes = 0, ok = 0;
  *probes_out = 0;
  *t_out = t;
  *dirchg_out = 0;
  if (!(e_b > 0.0)) return 0;
  uint8_t *Acand = (uint8_t *)malloc((size_t)s_it);
  for (;;) {
    /* Apply-Threshold: finished = rel-err finished or E_i < t; e_abar, the
     * error of the finished candidates, summed directly (e_it - sum(A.E) is
     * the same number formed by cancellation) */
    nsum fin = {0, 0};
    int64_t sumA = 0;
    for (int64_t i = 0; i < s_it; ++i) {
      Acand[i] = A[i] && !(E[i] < t);
      sumA += Acand[i];
      if (!Acand[i]) nadd(&fin, E[i]);
    }
    ++probes;
    int64_t s_abar = s_it - sumA;
    int dir;
    if (s_abar > 0.5 * (double)s_it) {           /* memory requirement */
      double e_abar = nval(&fin);
      if (e_abar <= Pmax * e_b) { ok = 1; break; } /* accuracy requirement */
      dir = -1;                                   /* too much error: lower t */
    } else {
      dir = +1;                                   /* too few finished: raise t */
    }
    if (last_dir != 0 && dir != last_dir) {
      ++changes;
      Pmax = fmin(Pmax + 0.10, 0.95);
    }
    last_dir = dir;
    if (changes >= 10 || probes >= 64) break;
    if (dir > 0) t = t + (mx - t) / 2.0;
    else t = t - (t - mn) / 2.0;
  }
  if (ok) memcpy(A, Acand, (size_t)s_it);
  free(Acand);
  *probes_out = probes;
  *t_out = t;
  *dirchg_out = changes;
  return ok;
}

/* ------------------------------------------------------- Uniform-Split ---- */
int oracle_default_init_div(int n) {
  int d = 2;
  while (1) {
    int64_t pw = 1;
    for (int j = 0; j < n; ++j) pw *= 2 * d;
    if (pw > 4096) break;
    d *= 2;
  }
  return d;
}

/* Region i of the d^n grid over [a, b] (a, b NULL: the unit cube): axis
 * n-1 varies fastest. */
static void uniform_split(int n, int d, const double *a, const double *b, double *lower,
                          double *width) {
  int64_t s = 1;
  for (int j = 0; j < n; ++j) s *= d;
  for (int64_t i = 0; i < s; ++i) {
    int64_t r = i;
    for (int j = n - 1; j >= 0; --j) {
      double a_j = a ? a[j] : 0.0, len = a ? b[j] - a[j] : 1.0;
      lower[i * n + j] = a_j + len * (double)(r % d) / (double)d;
      width[i * n + j] = len / (double)d;
      r /= d;
    }
  }
}

/* ------------------------------------------------------ PAGANI main loop -- */
/* Appends box i of (lo, wd) to the leaf list (row-major, capacity cap). */
static void leaf_append(int n, const double *lo, const double *wd, double *leaf_lo,
                        double *leaf_w, int64_t cap, int64_t *count) {
  if (leaf_lo && *count < cap) {
    memcpy(leaf_lo + *count * n, lo, sizeof(double) * n);
    memcpy(leaf_w + *count * n, wd, sizeof(double) * n);
  }
  ++*count;
}

int oracle_pagani(const oracle_rule *R, int fam, const double *params,
                  double tau_rel, double tau_abs, int64_t max_regions,
                  const oracle_options *opt, oracle_result *res,
                  oracle_trace *trace, int trace_cap,
                  double *final_lower, double *final_width, int64_t final_cap,
                  double *fin_vol_out, double *leaf_lo, double *leaf_w,
                  int64_t leaf_cap, int64_t *n_leaves) {
  int64_t leaves = 0;
  int n = R->n;
  int d = opt->init_div > 0 ? opt->init_div : oracle_default_init_div(n);
  int64_t s = 1;
  for (int j = 0; j < n; ++j) s *= d;
  memset(res, 0, sizeof(*res));
  if (s > max_regions) { res->status = -7; return -7; }
  if ((opt->lower == NULL) != (opt->upper == NULL)) { res->status = -8; return -8; }
  for (int j = 0; opt->lower && j < n; ++j)
    if (!(opt->upper[j] > opt->lower[j]) || !isfinite(opt->upper[j] - opt->lower[j])) {
      res->status = -8;
      return -8;
    }

  int64_t cap = s > max_regions ? s : max_regions;
  double *H_lo = (double *)malloc(sizeof(double) * (size_t)cap * n);
  double *H_w = (double *)malloc(sizeof(double) * (size_t)cap * n);
  double *V = (double *)calloc((size_t)cap, sizeof(double));
  double *E = (double *)calloc((size_t)cap, sizeof(double));
  int32_t *K = (int32_t *)calloc((size_t)cap, sizeof(int32_t));
  uint8_t *A = (uint8_t *)malloc((size_t)cap);
  double *Vp = (double *)calloc((size_t)cap, sizeof(double));
  double *Ep = (double *)calloc((size_t)cap, sizeof(double));
  double v = 0, e = 0, vf = 0, ef = 0, v_tot_prev = 0, tau_cls = tau_rel;
  nsum finvol = {0, 0};
  int status = 1, it;

  uniform_split(n, d, opt->lower, opt->upper, H_lo, H_w);   /* H <- Uniform-Split([a, b], d) */
  memset(A, 1, (size_t)s);                      /* A[1:s] <- 1 */

  for (it = 1; it <= opt->it_max; ++it) {
    oracle_trace tr;
    memset(&tr, 0, sizeof(tr));
    tr.it = it;
    tr.s = s;
    res->n_regions += s;
    res->n_active_last = s;
    /* V, E, K <- Evaluate(H).  Regions are independent: the second,
       OpenMP build of this file (the parallel CPU baseline) runs this loop
       on all host cores; every other step stays serial and in order. */
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < s; ++i) {
      int k;
      evaluate_region(R, fam, params, H_lo + i * n, H_w + i * n, &V[i], &E[i],
                      &k, NULL);
      K[i] = k;
    }
    for (int64_t i = 0; i < s; ++i)
      if (!isfinite(V[i]) || !isfinite(E[i])) { status = -6; goto done; }
    /* E <- Two-Level-Error(V, E, V_p, E_p) */
    if (it > 1) two_level_error(s, V, E, Vp);
    /* A <- Rel-Err-Classify(V, E, A), at the survivors' share tau_cls */
    rel_err_classify(s, V, E, tau_cls, opt->relerr_filter, A);
    /* v <- Sum(V); e <- Sum(E) */
    nsum sv = {0, 0}, se = {0, 0};
    for (int64_t i = 0; i < s; ++i) { nadd(&sv, V[i]); nadd(&se, E[i]); }
    v = nval(&sv);
    e = nval(&se);
    int64_t n_rel = 0;
    for (int64_t i = 0; i < s; ++i) n_rel += A[i];
    tr.v = v; tr.e = e; tr.vf = vf; tr.ef = ef;
    tr.n_relerr_active = n_rel;
    /* termination test */
    if ((e + ef) / fabs(v + vf) <= tau_rel || e + ef <= tau_abs) {
      status = 0;
      tr.n_survivors = 0;
      if (trace && it - 1 < trace_cap) trace[it - 1] = tr;
      break;
    }
    if (it == opt->it_max) {
      status = 1;
      if (trace && it - 1 < trace_cap) trace[it - 1] = tr;
      break;
    }
    /* A <- Threshold-Classify(A, E, v + v_f, e_f, e, s) when triggered */
    double v_tot = v + vf;
    int trig = 0;
    {
      int digits = opt->heuristic_filter == 1 || opt->heuristic_filter == 3;
      int memory = opt->heuristic_filter == 1 || opt->heuristic_filter == 2;
      if (digits && it >= 2 && fabs(v_tot - v_tot_prev) <= tau_rel * fabs(v_tot)) trig |= 1;
      if (memory && 2 * n_rel > max_regions) trig |= 2;
    }
    tr.trigger = trig;
    if (trig) {
      int probes, chg;
      double t;
      tr.search_ok = threshold_classify(A, E, v_tot, ef, e, s, tau_rel,
                                        &probes, &t, &chg);
      tr.probes = probes;
      tr.threshold = t;
      tr.direction_changes = chg;
    }
    v_tot_prev = v_tot;
    int64_t n_surv = 0;
    for (int64_t i = 0; i < s; ++i) n_surv += A[i];
    tr.n_survivors = n_surv;
    if (2 * n_surv > max_regions) {             /* memory exhausted */
      status = 2;
      if (trace && it - 1 < trace_cap) trace[it - 1] = tr;
      break;
    }
    /* v_f <- v - Sum(V.A) + v_f ; e_f <- e - Sum(E.A) + e_f, with v - Sum(V.A)
     * and e - Sum(E.A) summed directly over the finished regions */
    nsum svf = {0, 0}, sef = {0, 0};
    for (int64_t i = 0; i < s; ++i)
      if (!A[i]) { nadd(&svf, V[i]); nadd(&sef, E[i]); }
    double vf_new = vf + nval(&svf);
    double ef_new = ef + nval(&sef);
    tr.vf = vf_new; tr.ef = ef_new;
    if (trace && it - 1 < trace_cap) trace[it - 1] = tr;
    /* nothing left to refine: v + v_f and e + e_f cannot change any more,
     * so the loop ends as it would at it_max */
    if (n_surv == 0) {
      status = 1;
      break;
    }
    /* the survivors' share of what the tolerance still allows, rounded down
     * to a power of two */
    {
      double v_act = v - nval(&svf), allow = tau_rel * fabs(v + vf) - ef_new;
      tau_cls = tau_rel;
      if (allow < tau_rel * fabs(v_act)) {
        int ex;
        tau_cls = 0.0;
        if (allow > 0.0) {
          frexp(allow / fabs(v_act), &ex);
          tau_cls = ldexp(0.5, ex);
        }
      }
    }
    vf = vf_new;
    ef = ef_new;
    for (int64_t i = 0; i < s; ++i)
      if (!A[i]) {
        double vol = 1.0;
        for (int j = 0; j < n; ++j) vol *= H_w[i * n + j];
        nadd(&finvol, vol);
        /* finished boxes leave the list for good: they are leaves */
        leaf_append(n, H_lo + i * n, H_w + i * n, leaf_lo, leaf_w, leaf_cap, &leaves);
      }
    /* H, V, E <- Filter(H, V, E, A); V_p <- V, E_p <- E */
    int64_t q = 0;
    for (int64_t i = 0; i < s; ++i) {
      if (!A[i]) continue;
      memmove(H_lo + q * n, H_lo + i * n, sizeof(double) * n);
      memmove(H_w + q * n, H_w + i * n, sizeof(double) * n);
      Vp[q] = V[i];
      Ep[q] = E[i];
      K[q] = K[i];
      ++q;
    }
    /* H <- Split(H, K): children of p at 2p (lower) and 2p+1 (upper) */
    for (int64_t pp = q - 1; pp >= 0; --pp) {
      int k = K[pp];
      for (int j = 0; j < n; ++j) {
        double lo = H_lo[pp * n + j], w = H_w[pp * n + j];
        H_lo[(2 * pp) * n + j] = lo;
        H_w[(2 * pp) * n + j] = w;
        H_lo[(2 * pp + 1) * n + j] = lo;
        H_w[(2 * pp + 1) * n + j] = w;
      }
      H_w[(2 * pp) * n + k] *= 0.5;
      H_w[(2 * pp + 1) * n + k] *= 0.5;
      H_lo[(2 * pp + 1) * n + k] += H_w[(2 * pp + 1) * n + k];
    }
    s = 2 * q;                                  /* s <- 2s */
    memset(A, 1, (size_t)s);
  }
  if (it > opt->it_max) it = opt->it_max;
done:
  res->status = status;
  res->iterations = it;
  res->estimate = v + vf;
  res->errorest = e + ef;
  if (final_lower && final_width) {
    int64_t m = s < final_cap ? s : final_cap;
    memcpy(final_lower, H_lo, sizeof(double) * (size_t)m * n);
    memcpy(final_width, H_w, sizeof(double) * (size_t)m * n);
  }
  if (fin_vol_out) *fin_vol_out = nval(&finvol);
  /* every box of the last iteration is a leaf too */
  if (status >= 0)
    for (int64_t i = 0; i < s; ++i)
      leaf_append(n, H_lo + i * n, H_w + i * n, leaf_lo, leaf_w, leaf_cap, &leaves);
  if (n_leaves) *n_leaves = leaves;
  free(H_lo); free(H_w); free(V); free(E); free(K); free(A); free(Vp); free(Ep);
  return status;
}

/* Exported for unit tests of Threshold-Classify on synthetic error lists. */
int oracle_threshold_classify(uint8_t *A, const double *E, double v_tot,
                              double e_f, double e_it, int64_t s_it,
                              double tau_rel, int *probes, double *t,
                              int *direction_changes) {
  return threshold_classify(A, E, v_tot, e_f, e_it, s_it, tau_rel, probes, t,
                            direction_changes);
}


/* ------------------------------------------------------------- gradients -- */
/* Integrand and its derivatives with respect to the parameter vector
 * (family layout), written from the formulas: d[k] = df/dparams[k].
 * Defined for the product peak, Gaussian and C0 families. */
static double integrand_grad(int fam, int n, const double *p, const double *x,
                             double *d) {
  double f = integrand(fam, n, p, x);
  for (int j = 0; j < n; ++j) {
    double t = x[j] - p[n + j];
    switch (fam) {
    case FAM_PRODUCT_PEAK: { /* f = prod 1/(c^-2 + t^2) */
      double den = pow(p[j], -2.0) + t * t;
      d[j] = f * (2.0 * pow(p[j], -3.0)) / den;
      d[n + j] = f * (2.0 * t) / den;
      break;
    }
    case FAM_GAUSSIAN: /* f = exp(-sum a^2 t^2) */
      d[j] = f * (-2.0 * p[j] * t * t);
      d[n + j] = f * (2.0 * p[j] * p[j] * t);
      break;
    case FAM_C0: /* f = exp(-sum a |t|) */
      d[j] = f * (-fabs(t));
      d[n + j] = f * (t > 0.0 ? p[j] : (t < 0.0 ? -p[j] : 0.0));
      break;
    default:
      d[j] = d[n + j] = NAN;
    }
  }
  return f;
}

/* Sum over the boxes (row-major lower/width, m x n) of the basic rule
 * applied to f and to each df/dparams[k]: out[0] = sum V, out[1 + k] = sum
 * dV/dparams[k]; absout receives the same sums of absolute values (their
 * rounding scale). */
int oracle_gradient(const oracle_rule *R, int fam, const double *params,
                    int64_t m, const double *lower, const double *width,
                    double *out, double *absout) {
  int n = R->n, K = 2 * n + 1;
  nsum acc[17];
  double sab[17];
  memset(acc, 0, sizeof(acc));
  memset(sab, 0, sizeof(sab));
  for (int64_t i = 0; i < m; ++i) {
    double c[16], h[16], vol = 1.0;
    for (int j = 0; j < n; ++j) {
      h[j] = 0.5 * width[i * n + j];
      c[j] = lower[i * n + j] + h[j];
      vol *= width[i * n + j];
    }
    double box[17], boxab[17];
    memset(box, 0, sizeof(box));
    memset(boxab, 0, sizeof(boxab));
    for (int g = 0; g < R->G; ++g) {
      double wg = R->wts[g * 5];
      if (wg == 0.0) continue;
      double v[16], x[16], d[16];
      memcpy(v, R->gen + (size_t)g * n, sizeof(double) * n);
      qsort(v, n, sizeof(double), cmp_double);
      do {
        int nzi[16], nz = 0;
        for (int j = 0; j < n; ++j)
          if (v[j] != 0.0) nzi[nz++] = j;
        for (int mask = 0; mask < (1 << nz); ++mask) {
          for (int j = 0; j < n; ++j) x[j] = c[j];
          for (int t = 0; t < nz; ++t) {
            int j = nzi[t];
            x[j] = c[j] + h[j] * ((mask >> t & 1) ? -v[j] : v[j]);
          }
          double f = integrand_grad(fam, n, params, x, d);
          box[0] += wg * f;
          boxab[0] += fabs(wg * f);
          for (int k = 0; k < 2 * n; ++k) {
            box[1 + k] += wg * d[k];
            boxab[1 + k] += fabs(wg * d[k]);
          }
        }
      } while (next_perm(v, n));
    }
    for (int k = 0; k < K; ++k) {
      nadd(&acc[k], vol * box[k]);
      sab[k] += vol * boxab[k];
    }
  }
  for (int k = 0; k < K; ++k) {
    out[k] = nval(&acc[k]);
    if (absout) absout[k] = sab[k];
  }
  return 0;
}
