"""The identity behind the gradient kernel, checked on the CPU against
point-by-point enumeration.

For a product integrand, a box's basic-rule value V is multilinear in the
per-axis factor values t_j(c).  Summed over the signs of an orbit, the
non-centre factors enter as s_j(r) = t_j(r+) + t_j(r-).  So the centre,
one-axis, pair and triple orbit sums are coefficients of
prod_j (t0_j + z s_j(1) + y s_j(2) + x s_j(3)), and the vertices give
prod_j s_j(0).  The chain rule through the factor values then gives
dV/dtheta_j.  Here the orbits of the degree-9 rule (Sec. 3.2, the Genz-Malik
structure: centre, one axis at three radii, pairs at (r1, r1) and (r1, r2)
in both orders, triples at r1, all vertices at r0) are enumerated point by
point with random factor values, weights and factor derivatives.  The
polynomial form must give the same V and gradient to rounding.
"""
import itertools

import numpy as np
import pytest


def _points(n, w):
    """(weight, per-axis slot) of every rule point with a basic weight;
    slots: 0 centre, 1/2 r1+-, 3/4 r2+-, 5/6 r3+-, 7/8 r0+-."""
    yield w[0], (0,) * n
    for j in range(n):
        for g, (a, b) in zip((1, 2, 3), ((1, 2), (3, 4), (5, 6))):
            for c in (a, b):
                x = [0] * n
                x[j] = c
                yield w[g], tuple(x)
    for j, k in itertools.combinations(range(n), 2):
        for cj in (1, 2):
            for ck in (1, 2):
                x = [0] * n
                x[j], x[k] = cj, ck
                yield w[5], tuple(x)
        for a, b in (((1, 2), (3, 4)), ((3, 4), (1, 2))):
            for cj in a:
                for ck in b:
                    x = [0] * n
                    x[j], x[k] = cj, ck
                    yield w[6], tuple(x)
    for j, k, l in itertools.combinations(range(n), 3):
        for sg in itertools.product((1, 2), repeat=3):
            x = [0] * n
            x[j], x[k], x[l] = sg
            yield w[7], tuple(x)
    for sg in itertools.product((7, 8), repeat=n):
        yield w[8], tuple(sg)


def _brute(n, t, dt, w):
    V, G = 0.0, np.zeros(n)
    for wg, x in _points(n, w):
        f = np.prod([t[x[j], j] for j in range(n)])
        V += wg * f
        for j in range(n):
            G[j] += wg * f * dt[x[j], j] / t[x[j], j]
    return V, G


def _polynomial(n, t, dt, w):
    t0 = t[0]
    s1, s2, s3, s0 = t[1] + t[2], t[3] + t[4], t[5] + t[6], t[7] + t[8]
    P1, Pz, Py, Pzz = [1.0], [0.0], [0.0], [0.0]
    px = pzy = pzzz = 0.0
    for m in range(n):
        px = px * t0[m] + P1[m] * s3[m]
        pzy = pzy * t0[m] + Pz[m] * s2[m] + Py[m] * s1[m]
        pzzz = pzzz * t0[m] + Pzz[m] * s1[m]
        P1.append(P1[m] * t0[m])
        Pz.append(Pz[m] * t0[m] + P1[m] * s1[m])
        Py.append(Py[m] * t0[m] + P1[m] * s2[m])
        Pzz.append(Pzz[m] * t0[m] + Pz[m] * s1[m])
    H0 = np.array([w[8] * np.prod([s0[m] for m in range(n) if m != j]) for j in range(n)])
    V = (w[0] * P1[n] + w[1] * Pz[n] + w[2] * Py[n] + w[3] * px + w[5] * Pzz[n] + w[6] * pzy
         + w[7] * pzzz + w[8] * np.prod(s0))
    G = np.zeros(n)
    q1, qz, qy, qzz = 1.0, 0.0, 0.0, 0.0
    for j in range(n - 1, -1, -1):
        L1 = P1[j] * q1
        Lz = P1[j] * qz + Pz[j] * q1
        Ly = P1[j] * qy + Py[j] * q1
        Lzz = P1[j] * qzz + Pz[j] * qz + Pzz[j] * q1
        H = [w[1] * L1 + w[5] * Lz + w[6] * Ly + w[7] * Lzz, w[2] * L1 + w[6] * Lz, w[3] * L1, H0[j]]
        for i in range(4):
            G[j] += (dt[2 * i + 1, j] + dt[2 * i + 2, j]) * H[i]
        gc = V - (s1[j] * H[0] + s2[j] * H[1] + s3[j] * H[2] + s0[j] * H[3])
        G[j] += dt[0, j] / t[0, j] * gc
        q1, qz, qy, qzz = q1 * t0[j], qz * t0[j] + q1 * s1[j], qy * t0[j] + q1 * s2[j], qzz * t0[j] + qz * s1[j]
    return V, G


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6])
def test_polynomial_form_matches_point_enumeration(n):
    rng = np.random.default_rng(100 + n)
    t = rng.uniform(0.5, 1.5, size=(9, n))
    dt = rng.normal(size=(9, n))
    w = rng.normal(size=9)
    w[4] = 0.0  # the lambda_p orbit carries no basic weight
    Vb, Gb = _brute(n, t, dt, w)
    Vp, Gp = _polynomial(n, t, dt, w)
    assert abs(Vp - Vb) <= 1e-13 * abs(Vb)
    assert np.max(np.abs(Gp - Gb)) <= 1e-13 * np.max(np.abs(Gb))


def test_polynomial_form_catches_a_dropped_orbit():
    """Zeroing one orbit's weight on one side only must show: the check is
    sensitive to every orbit."""
    n = 4
    rng = np.random.default_rng(7)
    t = rng.uniform(0.5, 1.5, size=(9, n))
    dt = rng.normal(size=(9, n))
    w = rng.normal(size=9)
    w[4] = 0.0
    Vb, _ = _brute(n, t, dt, w)
    for g in (0, 1, 2, 3, 5, 6, 7, 8):
        w2 = w.copy()
        w2[g] = 0.0
        Vp, _ = _polynomial(n, t, dt, w2)
        assert abs(Vp - Vb) > 1e-9 * abs(Vb)
