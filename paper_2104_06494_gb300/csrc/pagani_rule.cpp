// Degree-9 fully symmetric cubature rule with four null rules (and the
// Genz-Malik degree-7 variant), generated on the host in long double.
//
// The paper fixes the rule family (Sec. 2.1: the Genz-Malik rules used by
// Cuhre, 2^n + Theta(n^3) points; Sec. 3.2: four extra rules whose
// differences give the error).  It prints no constants, so the construction
// is this reading of them:
//  * squared radii l0 = 0.4707, l1 = 4/(15 - 5/l0), rho = (1 - l1/l0)/27,
//    l2 = (5 - 7 l1 - 35 rho)/(7 - 35 l1/3 - 35 rho/l0), rho' = rho (1 - l2/l0)/3,
//    l3 = (7 - 9(l2+l1) + 63 l2 l1/5 - 63 rho')/(9 - 63(l2+l1)/5 + 21 l2 l1 - 63 rho'/l0),
//    lp = 1/16;
//  * nine generator orbits: centre; one axis at l1, l2, l3, lp; axis pairs
//    (l1,l1) and (l1,l2); axis triples (l1,l1,l1); all axes at l0;
//  * basic weights solve the fully symmetric moment equations of degree <= 9
//    (least squares by Householder QR, residual checked);
//  * null rule k (degree 7, 5, 3, 1) = basic weights projected onto the null
//    space of the moment equations of that degree (count-weighted inner
//    product), orthogonalised against the previous null rules and scaled to
//    the basic rule's norm.
// Orbit moment sums are written in closed form per generator type.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "pagani_internal.h"

namespace pg {
namespace {

typedef long double ld;

struct Lambdas { ld l0, l1, l2, l3, lp; };

Lambdas make_lambdas() {
  Lambdas L;
  L.l0 = 0.4707L;
  L.l1 = 4.0L / (15.0L - 5.0L / L.l0);
  ld rho = (1.0L - L.l1 / L.l0) / 27.0L;
  L.l2 = (5.0L - 7.0L * L.l1 - 35.0L * rho) / (7.0L - 35.0L * L.l1 / 3.0L - 35.0L * rho / L.l0);
  ld rho2 = rho * (1.0L - L.l2 / L.l0) / 3.0L;
  L.l3 = (7.0L - 9.0L * (L.l2 + L.l1) + 63.0L * L.l2 * L.l1 / 5.0L - 63.0L * rho2) /
         (9.0L - 63.0L * (L.l2 + L.l1) / 5.0L + 21.0L * L.l2 * L.l1 - 63.0L * rho2 / L.l0);
  L.lp = 0.0625L;
  return L;
}

ld ipow(ld x, int e) { ld r = 1.0L; for (int i = 0; i < e; ++i) r *= x; return r; }
ld binom(int n, int k) {
  if (k < 0 || k > n) return 0.0L;
  ld r = 1.0L;
  for (int i = 0; i < k; ++i) r = r * (n - i) / (i + 1);
  return r;
}

// Fully symmetric moment condition: monomial prod_{i<m} x_i^(2 p_i) with
// parts p_0 >= ... >= p_{m-1} > 0 placed on the first m axes.
struct Part { int m; int p[4]; };

void partitions_rec(int k, int maxparts, int maxpart, Part cur, std::vector<Part>& out) {
  if (k == 0) { out.push_back(cur); return; }
  if (maxparts == 0) return;
  for (int first = (k < maxpart ? k : maxpart); first >= 1; --first) {
    Part nx = cur;
    nx.p[nx.m++] = first;
    partitions_rec(k - first, maxparts - 1, first, nx, out);
  }
}

std::vector<Part> moment_set(int n, int max_half_degree) {
  std::vector<Part> out;
  for (int k = 0; k <= max_half_degree; ++k) {
    Part z; z.m = 0; std::memset(z.p, 0, sizeof(z.p));
    partitions_rec(k, n < 4 ? n : 4, k, z, out);
  }
  return out;
}

// Sum over the orbit of generator g of the monomial, in closed form.
ld orbit_moment(int n, int g, const Part& P, const Lambdas& L) {
  const int m = P.m;
  int tot = 0;
  for (int i = 0; i < m; ++i) tot += P.p[i];
  switch (g) {
    case kGenCentre: return m == 0 ? 1.0L : 0.0L;
    case kGenL1: case kGenL2: case kGenL3: case kGenLp: {
      ld lam = g == kGenL1 ? L.l1 : g == kGenL2 ? L.l2 : g == kGenL3 ? L.l3 : L.lp;
      if (m == 0) return 2.0L * n;
      if (m == 1) return 2.0L * ipow(lam, P.p[0]);
      return 0.0L;
    }
    case kGenL1L1: {  // unordered axis pairs, both at l1, 4 signs
      if (m == 0) return 4.0L * binom(n, 2);
      if (m == 1) return 4.0L * (n - 1) * ipow(L.l1, P.p[0]);
      if (m == 2) return 4.0L * ipow(L.l1, P.p[0] + P.p[1]);
      return 0.0L;
    }
    case kGenL1L2: {  // ordered axis pairs (l1 on one, l2 on the other), 4 signs
      if (m == 0) return 4.0L * n * (n - 1);
      if (m == 1) return 4.0L * (n - 1) * (ipow(L.l1, P.p[0]) + ipow(L.l2, P.p[0]));
      if (m == 2) return 4.0L * (ipow(L.l1, P.p[0]) * ipow(L.l2, P.p[1]) + ipow(L.l2, P.p[0]) * ipow(L.l1, P.p[1]));
      return 0.0L;
    }
    case kGenL1L1L1: {  // unordered axis triples at l1, 8 signs
      if (n < 3) return 0.0L;
      if (m == 0) return 8.0L * binom(n, 3);
      if (m == 1) return 8.0L * binom(n - 1, 2) * ipow(L.l1, P.p[0]);
      if (m == 2) return 8.0L * (n - 2) * ipow(L.l1, P.p[0] + P.p[1]);
      if (m == 3) return 8.0L * ipow(L.l1, tot);
      return 0.0L;
    }
    case kGenL0All: return std::ldexp(1.0L, n) * ipow(L.l0, tot);
  }
  return 0.0L;
}

ld exact_moment(const Part& P) {
  ld r = 1.0L;
  for (int i = 0; i < P.m; ++i) r /= (2 * P.p[i] + 1);
  return r;
}

// Least-squares solution of the R x G system A x = b (R >= G, full column
// rank) by Householder QR.
bool lsq_qr(std::vector<ld> A, std::vector<ld> b, int R, int G, std::vector<ld>& x) {
  for (int k = 0; k < G; ++k) {
    ld norm = 0.0L;
    for (int r = k; r < R; ++r) norm += A[r * G + k] * A[r * G + k];
    norm = sqrtl(norm);
    if (norm == 0.0L) return false;
    const ld alpha = A[k * G + k] > 0 ? -norm : norm;
    std::vector<ld> v(R, 0.0L);
    for (int r = k; r < R; ++r) v[r] = A[r * G + k];
    v[k] -= alpha;
    ld vn = 0.0L;
    for (int r = k; r < R; ++r) vn += v[r] * v[r];
    if (vn == 0.0L) continue;
    for (int c = k; c < G; ++c) {
      ld d = 0.0L;
      for (int r = k; r < R; ++r) d += v[r] * A[r * G + c];
      d = 2.0L * d / vn;
      for (int r = k; r < R; ++r) A[r * G + c] -= d * v[r];
    }
    ld d = 0.0L;
    for (int r = k; r < R; ++r) d += v[r] * b[r];
    d = 2.0L * d / vn;
    for (int r = k; r < R; ++r) b[r] -= d * v[r];
  }
  x.assign(G, 0.0L);
  for (int r = G - 1; r >= 0; --r) {
    ld acc = b[r];
    for (int c = r + 1; c < G; ++c) acc -= A[r * G + c] * x[c];
    if (A[r * G + r] == 0.0L) return false;
    x[r] = acc / A[r * G + r];
  }
  return true;
}

}  // namespace

int64_t orbit_count(int n, int g) {
  switch (g) {
    case kGenCentre: return 1;
    case kGenL1: case kGenL2: case kGenL3: case kGenLp: return 2 * n;
    case kGenL1L1: return 2LL * n * (n - 1);
    case kGenL1L2: return 4LL * n * (n - 1);
    case kGenL1L1L1: return n >= 3 ? 4LL * n * (n - 1) * (n - 2) / 3 : 0;
    case kGenL0All: return 1LL << n;
  }
  return 0;
}

int num_points(int n) {
  int64_t t = 0;
  for (int g = 0; g < kNumGen; ++g) t += orbit_count(n, g);
  return (int)t;
}

// Weights of the orbits `gens` solving the moment equations of degree
// <= 2 half_degree + 1: least squares by Householder QR (no squaring of the
// condition number), then one refinement step on the residual of the
// original system.  Returns false if the system is rank deficient.
static bool solve_weights(int n, const std::vector<int>& gens, int half_degree, const Lambdas& L, std::vector<ld>& w,
                   ld* maxres_out) {
  const int G = (int)gens.size();
  std::vector<Part> rows = moment_set(n, half_degree);
  const int R = (int)rows.size();
  std::vector<ld> S(R * G), b(R);
  for (int r = 0; r < R; ++r) {
    for (int c = 0; c < G; ++c) S[r * G + c] = orbit_moment(n, gens[c], rows[r], L);
    b[r] = exact_moment(rows[r]);
  }
  if (!lsq_qr(S, b, R, G, w)) return false;
  {
    std::vector<ld> res(R), dw;
    for (int r = 0; r < R; ++r) {
      ld acc = b[r];
      for (int c = 0; c < G; ++c) acc -= S[r * G + c] * w[c];
      res[r] = acc;
    }
    if (lsq_qr(S, res, R, G, dw))
      for (int c = 0; c < G; ++c) w[c] += dw[c];
  }
  ld maxres = 0.0L;
  for (int r = 0; r < R; ++r) {
    ld s = -b[r];
    for (int c = 0; c < G; ++c) s += S[r * G + c] * w[c];
    maxres = fmaxl(maxres, fabsl(s) / b[r]);
  }
  if (maxres_out) *maxres_out = maxres;
  return true;
}

// Genz-Malik degree-7 rule with its embedded degree-5 rule, placed on the
// degree-9 generator slots that have its structure: centre; one axis at
// sqrt(9/70) (slot lp, the small fourth-difference radius); one axis at
// sqrt(9/10) (slot l2, the large one); two axes at sqrt(9/10) (slot l1l1,
// so l1 = 9/10); every axis at sqrt(9/19) (slot l0).  Weights from the moment
// equations of degree <= 7 (all five orbits) and <= 5 (the first four);
// null rule 1 = w7 - w5, the rule's error |R7 - R5|; null rules 2..4 unused.
static bool build_rule_gm7(int n, RuleTable* out, double* max_residual) {
  Lambdas L;
  L.l1 = L.l2 = L.l3 = 9.0L / 10.0L;
  L.lp = 9.0L / 70.0L;
  L.l0 = 9.0L / 19.0L;
  const std::vector<int> g7 = {kGenCentre, kGenLp, kGenL2, kGenL1L1, kGenL0All};
  const std::vector<int> g5 = {kGenCentre, kGenLp, kGenL2, kGenL1L1};
  std::vector<ld> w7, w5;
  ld r7 = 0.0L, r5 = 0.0L;
  if (!solve_weights(n, g7, 3, L, w7, &r7) || !solve_weights(n, g5, 2, L, w5, &r5)) return false;
  if (max_residual) *max_residual = (double)fmaxl(r7, r5);
  w5.push_back(0.0L);
  std::memset(out, 0, sizeof(*out));
  out->n = n;
  out->degree = 7;
  out->radius[0] = (double)sqrtl(L.l1);
  out->radius[1] = (double)sqrtl(L.l2);
  out->radius[2] = (double)sqrtl(L.l3);
  out->radius[3] = (double)sqrtl(L.lp);
  out->radius[4] = (double)sqrtl(L.l0);
  out->q = (double)(L.lp / L.l2);
  int64_t pts = 0;
  for (int c = 0; c < 5; ++c) {
    const int g = g7[c];
    out->count[g] = orbit_count(n, g);
    pts += out->count[g];
    out->w[g][0] = (double)w7[c];
    out->w[g][1] = (double)(w7[c] - w5[c]);
  }
  out->num_points = (int)pts;
  return true;
}

bool build_rule(int n, int degree, RuleTable* out, double* max_residual) {
  if (n < 2 || n > kMaxDim) return false;
  if (degree == 7) return build_rule_gm7(n, out, max_residual);
  if (degree != 9) return false;
  const Lambdas L = make_lambdas();
  std::vector<int> gens;
  for (int g = 0; g < kNumGen; ++g) if (orbit_count(n, g) > 0) gens.push_back(g);
  const int G = (int)gens.size();

  // basic rule: the degree-9 moment equations
  std::vector<ld> w;
  ld maxres = 0.0L;
  if (!solve_weights(n, gens, 4, L, w, &maxres)) return false;
  if (max_residual) *max_residual = (double)maxres;

  // count-weighted inner product <a, c> = sum_g cnt_g a_g c_g
  std::vector<ld> cnt(G);
  for (int c = 0; c < G; ++c) cnt[c] = (ld)orbit_count(n, gens[c]);
  auto inner = [&](const std::vector<ld>& a, const std::vector<ld>& c) {
    ld s = 0.0L;
    for (int g = 0; g < G; ++g) s += cnt[g] * a[g] * c[g];
    return s;
  };
  const ld wnorm = sqrtl(inner(w, w));

  // null rules of degree 7, 5, 3, 1
  const int degrees[4] = {7, 5, 3, 1};
  std::vector<std::vector<ld>> nulls;
  for (int k = 0; k < 4; ++k) {
    std::vector<Part> crow = moment_set(n, (degrees[k] - 1) / 2);
    // constraint sum_g S_g a_g = 0 is <M^-1 S, a> = 0: orthonormalise the
    // vectors M^-1 S (modified Gram-Schmidt, dropping dependent ones) and
    // remove their span from w
    std::vector<std::vector<ld>> basis;
    for (const Part& P : crow) {
      std::vector<ld> v(G);
      for (int g = 0; g < G; ++g) v[g] = orbit_moment(n, gens[g], P, L) / cnt[g];
      ld n0 = sqrtl(inner(v, v));
      for (int pass = 0; pass < 2; ++pass)
        for (auto& e : basis) {
          ld c = inner(v, e);
          for (int g = 0; g < G; ++g) v[g] -= c * e[g];
        }
      ld nv = sqrtl(inner(v, v));
      if (nv <= 1e-12L * n0) continue;
      for (int g = 0; g < G; ++g) v[g] /= nv;
      basis.push_back(v);
    }
    std::vector<ld> u = w;
    for (int pass = 0; pass < 2; ++pass)
      for (auto& e : basis) {
        ld c = inner(u, e);
        for (int g = 0; g < G; ++g) u[g] -= c * e[g];
      }
    for (int pass = 0; pass < 2; ++pass)
      for (auto& prev : nulls) {
        ld c = inner(u, prev) / inner(prev, prev);
        for (int g = 0; g < G; ++g) u[g] -= c * prev[g];
      }
    ld un = sqrtl(inner(u, u));
    if (!(un > 0.0L)) return false;
    for (int g = 0; g < G; ++g) u[g] *= wnorm / un;
    nulls.push_back(u);
  }

  std::memset(out, 0, sizeof(*out));
  out->n = n;
  out->degree = 9;
  out->radius[0] = (double)sqrtl(L.l1);
  out->radius[1] = (double)sqrtl(L.l2);
  out->radius[2] = (double)sqrtl(L.l3);
  out->radius[3] = (double)sqrtl(L.lp);
  out->radius[4] = (double)sqrtl(L.l0);
  // fourth-difference weights: the two inner radii (sqrt(lp), sqrt(l2)) and
  // the inner and outer radius (sqrt(l2), sqrt(l1))
  out->q = (double)(L.lp / L.l2);
  out->q_outer = (double)(L.l2 / L.l1);
  for (int c = 0; c < G; ++c) {
    int g = gens[c];
    out->count[g] = orbit_count(n, g);
    out->w[g][0] = (double)w[c];
    for (int k = 0; k < 4; ++k) out->w[g][1 + k] = (double)nulls[k][c];
  }
  out->num_points = num_points(n);
  return true;
}

}  // namespace pg

namespace pg {

// Every rule point of dimension n as a packed word: bits 4j..4j+3 hold the
// coordinate code (Code enum) of axis j, bits 32..35 the generator orbit.
// Orbits are enumerated from their structure: axes chosen in increasing
// order, every sign pattern.
std::vector<uint64_t> point_codes(int n) {
  std::vector<uint64_t> out;
  auto emit = [&](int g, const int* axes, const int* codes, int k) {
    uint64_t w = (uint64_t)g << 32;
    for (int t = 0; t < k; ++t) w |= (uint64_t)codes[t] << (4 * axes[t]);
    out.push_back(w);
  };
  const int one_axis_gen[4] = {kGenL1, kGenL2, kGenL3, kGenLp};
  const int one_axis_code[4] = {kR1P, kR2P, kR3P, kRpP};
  emit(kGenCentre, nullptr, nullptr, 0);
  for (int g = 0; g < 4; ++g)
    for (int j = 0; j < n; ++j)
      for (int sgn = 0; sgn < 2; ++sgn) {
        int axes[1] = {j}, codes[1] = {one_axis_code[g] + sgn};
        emit(one_axis_gen[g], axes, codes, 1);
      }
  for (int j = 0; j < n; ++j)
    for (int k = j + 1; k < n; ++k)
      for (int s = 0; s < 4; ++s) {
        int axes[2] = {j, k}, codes[2] = {kR1P + (s & 1), kR1P + (s >> 1)};
        emit(kGenL1L1, axes, codes, 2);
      }
  for (int j = 0; j < n; ++j)
    for (int k = 0; k < n; ++k) {
      if (j == k) continue;
      for (int s = 0; s < 4; ++s) {
        int axes[2] = {j, k}, codes[2] = {kR1P + (s & 1), kR2P + (s >> 1)};
        emit(kGenL1L2, axes, codes, 2);
      }
    }
  for (int j = 0; j < n; ++j)
    for (int k = j + 1; k < n; ++k)
      for (int l = k + 1; l < n; ++l)
        for (int s = 0; s < 8; ++s) {
          int axes[3] = {j, k, l}, codes[3] = {kR1P + (s & 1), kR1P + ((s >> 1) & 1), kR1P + (s >> 2)};
          emit(kGenL1L1L1, axes, codes, 3);
        }
  for (int s = 0; s < (1 << n); ++s) {
    int axes[8], codes[8];
    for (int j = 0; j < n; ++j) {
      axes[j] = j;
      codes[j] = kR0P + ((s >> j) & 1);
    }
    emit(kGenL0All, axes, codes, n);
  }
  return out;
}

}  // namespace pg
