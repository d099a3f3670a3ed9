"""Pins of the CPU oracle against facts fixed by the mathematics and the paper.

None of these checks re-evaluates the oracle's own formulas.  Each one holds for
an independent reason -- a closed form (shell theorem, binomial series), an
identity (force = -grad of the potential energy, exactness of re-expanding a
polynomial, Laplace's equation), an invariant (momentum, coverage) or brute
force -- chosen so that a dropped term, a wrong sign or index, or a transposed
operand in the oracle fails at least one of them.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1609_08621_gb300 import synth

MI = oracle.multi_index()


def _idx(a, b, c):
    hits = np.where((MI[:, 0] == a) & (MI[:, 1] == b) & (MI[:, 2] == c))[0]
    return int(hits[0])


# ---------------------------------------------------------------- direct sum


def test_direct_force_is_minus_gradient_of_potential_energy():
    """a_i = -(1/m_i) dU/dx_i with U = 1/2 sum_i m_i phi_i (finite differences of the oracle's pot)."""
    rng = np.random.default_rng(11)
    n = 7
    pos = rng.random((3, n))
    mass = 0.5 + rng.random(n)
    eps = 0.05
    acc, _ = oracle.direct(pos, mass, eps)

    def energy(p):
        _, ph = oracle.direct(p, mass, eps)
        return 0.5 * math.fsum(mass * ph)

    h = 1e-5
    for i in range(n):
        for a in range(3):
            pp, pm = pos.copy(), pos.copy()
            pp[a, i] += h
            pm[a, i] -= h
            g = (energy(pp) - energy(pm)) / (2 * h)
            assert abs(-g / mass[i] - acc[a, i]) <= 1e-6 * (1 + abs(acc[a, i]))


def test_direct_two_body_newton():
    """Two softened point masses: |a| = m d / (d^2+eps^2)^(3/2), attractive, phi = -m/sqrt(d^2+eps^2)."""
    d, eps = 0.3, 0.01
    pos = np.array([[0.2, 0.2 + d], [0.5, 0.5], [0.5, 0.5]])
    mass = np.array([2.0, 3.0])
    acc, pot = oracle.direct(pos, mass, eps)
    s = (d * d + eps * eps) ** 1.5
    assert acc[0, 0] == pytest.approx(3.0 * d / s, rel=1e-14)
    assert acc[0, 1] == pytest.approx(-2.0 * d / s, rel=1e-14)
    assert np.all(np.abs(acc[1:]) < 1e-18)
    assert pot[0] == pytest.approx(-3.0 / math.sqrt(d * d + eps * eps), rel=1e-14)
    assert pot[1] == pytest.approx(-2.0 / math.sqrt(d * d + eps * eps), rel=1e-14)


@pytest.mark.parametrize("n", [3, 5, 8])
def test_direct_tiny_n_against_extended_precision(n):
    """N <= 8 summed term by term in 40-digit arithmetic: the FP64 sums agree to a few ulp."""
    mpmath = pytest.importorskip("mpmath")
    rng = np.random.default_rng(100 + n)
    pos = rng.random((3, n))
    mass = 0.2 + rng.random(n)
    eps = 0.01
    acc, pot = oracle.direct(pos, mass, eps)
    with mpmath.workdps(40):
        P = [[mpmath.mpf(float(v)) for v in row] for row in pos]
        M = [mpmath.mpf(float(v)) for v in mass]
        e2 = mpmath.mpf(eps) ** 2
        for i in range(n):
            a = [mpmath.mpf(0)] * 3
            ph = mpmath.mpf(0)
            for j in range(n):
                if j == i:
                    continue
                d = [P[q][j] - P[q][i] for q in range(3)]
                R = mpmath.sqrt(d[0] ** 2 + d[1] ** 2 + d[2] ** 2 + e2)
                for q in range(3):
                    a[q] += M[j] * d[q] / R ** 3
                ph -= M[j] / R
            for q in range(3):
                assert acc[q, i] == pytest.approx(float(a[q]), rel=1e-14, abs=1e-14 * float(mpmath.fabs(ph)))
            assert pot[i] == pytest.approx(float(ph), rel=1e-15)


def test_direct_momentum_translation_linearity_scaling():
    pos, mass = synth.clustered_plummer(600, 5)
    mass = mass.astype(np.float64) * (1 + np.arange(600) % 3)
    eps = 1e-3
    acc, pot = oracle.direct(pos, mass, eps)
    # momentum: sum_i m_i a_i = 0 (pair antisymmetry)
    mom = (mass * acc).sum(axis=1)
    assert np.all(np.abs(mom) <= 1e-12 * (mass * np.abs(acc)).sum())
    # translation invariance
    acc2, pot2 = oracle.direct(pos + np.array([[0.125], [-0.25], [0.0625]]), mass, eps)
    assert np.allclose(acc2, acc, rtol=1e-9, atol=1e-9 * np.abs(acc).max())
    # linearity in the masses
    acc3, _ = oracle.direct(pos, 2.5 * mass, eps)
    assert np.allclose(acc3, 2.5 * acc, rtol=1e-13)
    # scaling: x -> s x, eps -> s eps gives a -> a / s^2, phi -> phi / s
    s = 0.5
    acc4, pot4 = oracle.direct(s * pos, mass, s * eps)
    assert np.allclose(acc4, acc / s ** 2, rtol=1e-10)
    assert np.allclose(pot4, pot / s, rtol=1e-12)


def _lattice_sphere(nside, radius=0.25, centre=0.5):
    g = (np.arange(nside) - (nside - 1) / 2.0) * (2.0 * radius / nside)
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    keep = X ** 2 + Y ** 2 + Z ** 2 <= radius ** 2
    pts = np.stack([X[keep], Y[keep], Z[keep]]) + centre
    return pts, 2.0 * radius / nside


@pytest.mark.parametrize("nside", [36, 56])
def test_uniform_sphere_shell_theorem(nside):
    """Uniform sphere (lattice clipped to the sphere, cubic symmetry), zero-mass probes.

    Exterior: |a| = M / r^2 (Newton's shell theorem; the lattice has cubic symmetry so
    its first non-zero multipole beyond the monopole is l = 4).  Interior: |a| = M r / R^3.
    """
    R, c = 0.25, 0.5
    pts, h = _lattice_sphere(nside, R, c)
    n = pts.shape[1]
    M = 1.0
    dirs = np.array([[0.48, 0.6, 0.64], [-0.36, 0.8, -0.48], [0.0, -0.6, 0.8]]).T
    dirs = dirs / np.linalg.norm(dirs, axis=0)
    r_ext = np.array([2.0 * R, 3.0 * R])
    r_int = np.array([0.5 * R])
    probes = []
    for r in np.concatenate([r_ext, r_int]):
        probes.append(c + r * dirs)
    probes = np.concatenate(probes, axis=1)
    pos = np.concatenate([pts, probes], axis=1)
    mass = np.concatenate([np.full(n, M / n), np.zeros(probes.shape[1])])
    sinks = np.arange(n, pos.shape[1])
    # exterior: negligible softening; interior: softening of one lattice spacing smooths granularity
    acc_e, _ = oracle.direct(pos, mass, 1e-7, sinks[: 2 * dirs.shape[1]])
    acc_i, _ = oracle.direct(pos, mass, h, sinks[2 * dirs.shape[1]:])
    k = dirs.shape[1]
    for j, r in enumerate(r_ext):
        a = acc_e[:, j * k:(j + 1) * k]
        radial = -(a * dirs).sum(axis=0)
        assert np.all(np.abs(radial / (M / r ** 2) - 1) < 2e-3)
        assert np.all(np.linalg.norm(a + radial * dirs, axis=0) < 2e-3 * M / r ** 2)
    a = acc_i
    radial = -(a * dirs).sum(axis=0)
    expect = M * r_int[0] / R ** 3
    assert np.all(np.abs(radial / expect - 1) < 1.5e-2)


# ---------------------------------------------------------------- expansion operators


def test_green_derivs_against_finite_differences_and_closed_forms():
    r = np.array([0.31, -0.17, 0.23])
    eps2 = 0.02 ** 2
    D = oracle.green_derivs(r, eps2)
    R2 = r @ r + eps2
    assert D[0] == pytest.approx(R2 ** -0.5, rel=1e-15)
    # first derivatives: -r / R^3
    assert np.allclose(D[1:4], -r / R2 ** 1.5, rtol=1e-14)
    # each derivative is the finite difference of the next lower order
    h = 1e-5
    for i in range(oracle.NMI):
        a, b, c = MI[i]
        if a + b + c >= 5:
            continue
        for ax in range(3):
            e = np.zeros(3)
            e[ax] = h
            fd = (oracle.green_derivs(r + e, eps2)[i] - oracle.green_derivs(r - e, eps2)[i]) / (2 * h)
            up = [a, b, c]
            up[ax] += 1
            assert abs(fd - D[_idx(*up)]) <= 1e-6 * (1 + abs(D[_idx(*up)]))


def test_green_derivs_laplacian():
    """Plummer: lap G = -3 eps^2 / R^5.  eps = 0: every trace vanishes (harmonic)."""
    r = np.array([0.21, 0.13, -0.37])
    for eps2 in (0.0, 0.05 ** 2):
        D = oracle.green_derivs(r, eps2)
        R2 = r @ r + eps2
        lap = D[_idx(2, 0, 0)] + D[_idx(0, 2, 0)] + D[_idx(0, 0, 2)]
        assert lap == pytest.approx(-3 * eps2 / R2 ** 2.5, abs=1e-12 * abs(D[_idx(2, 0, 0)]))
        if eps2 == 0.0:
            for i in range(oracle.NMI):
                a, b, c = MI[i]
                if a + b + c > 3:
                    continue
                tr = D[_idx(a + 2, b, c)] + D[_idx(a, b + 2, c)] + D[_idx(a, b, c + 2)]
                assert abs(tr) <= 1e-11 * np.abs(D).max()


def test_p2m_parallel_axis_identity():
    """Moments about c+t follow from moments about c by the binomial theorem."""
    rng = np.random.default_rng(3)
    pos = rng.random((3, 9))
    mass = rng.random(9)
    c = np.array([0.4, 0.5, 0.6])
    t = np.array([0.05, -0.02, 0.03])
    M0 = oracle.p2m(pos, mass, c)
    M1 = oracle.p2m(pos, mass, c + t)
    for i in range(oracle.NM4):
        n = MI[i]
        s = 0.0
        for j in range(oracle.NM4):
            k = MI[j]
            if np.all(k <= n):
                binom = np.prod([math.comb(int(n[q]), int(k[q])) for q in range(3)])
                s += binom * np.prod((-t) ** (n - k)) * M0[j]
        assert s == pytest.approx(M1[i], rel=1e-10, abs=1e-14)
    assert M0[0] == pytest.approx(mass.sum())


def test_m2p_single_particle_equals_pp():
    x = np.array([0.1, 0.2, 0.3])
    z = np.array([0.6, 0.5, 0.4])
    M = oracle.p2m(z.reshape(3, 1), np.array([0.7]), z)
    acc, pot = oracle.m2p(M, z, x, 1e-4)
    ref, rp = oracle.direct(np.stack([x, z], axis=1), np.array([0.0, 0.7]), 1e-2, [0])
    assert np.allclose(acc, ref[:, 0], rtol=1e-14)
    assert pot == pytest.approx(rp[0], rel=1e-14)


def test_m2p_error_decays_as_fifth_power():
    """Order-4 moments: the first neglected term is order 5, so the force error ~ (b/d)^5 |a|."""
    rng = np.random.default_rng(5)
    k = 40
    cl = 0.02 * (rng.random((3, k)) - 0.5)
    m = rng.random(k)
    com = (cl * m).sum(axis=1) / m.sum()
    cl = cl - com[:, None] + 0.5
    z = np.full(3, 0.5)
    M = oracle.p2m(cl, m, z)
    dirn = np.array([0.6, 0.48, 0.64])
    errs = []
    ds = np.array([0.08, 0.16, 0.32])
    for d in ds:
        x = z + d * dirn
        acc, _ = oracle.m2p(M, z, x, 0.0)
        ref, _ = oracle.direct(np.concatenate([cl, x[:, None]], axis=1), np.append(m, 0.0), 0.0, [k])
        errs.append(np.linalg.norm(acc - ref[:, 0]) / np.linalg.norm(ref[:, 0]))
    slope = np.polyfit(np.log(ds), np.log(errs), 1)[0]
    assert -6.2 < slope < -4.8


def test_m2p_binomial_series_two_masses():
    """eps = 0, masses m at z0 +- a e_z: potential on the axis is m/(s-a) + m/(s+a).
    Moments to order 4 reproduce 2m/s (1 + a^2/s^2 + a^4/s^4) exactly."""
    a, m, s = 0.03, 0.5, 0.2
    z0 = np.array([0.5, 0.5, 0.5])
    pos = np.stack([z0 + [0, 0, a], z0 - [0, 0, a]], axis=1)
    M = oracle.p2m(pos, np.array([m, m]), z0)
    acc, pot = oracle.m2p(M, z0, z0 + [0, 0, s], 0.0)
    assert -pot == pytest.approx(2 * m / s * (1 + a ** 2 / s ** 2 + a ** 4 / s ** 4), rel=1e-13)
    # force along the axis: derivative of the truncated series
    fz = -2 * m * (1 / s ** 2 + 3 * a ** 2 / s ** 4 + 5 * a ** 4 / s ** 6)
    assert acc[2] == pytest.approx(fz, rel=1e-12)
    assert abs(acc[0]) < 1e-14 and abs(acc[1]) < 1e-14


def test_l2l_is_exact_reexpansion():
    """A local expansion is a polynomial of degree 5: shifting it is exact."""
    rng = np.random.default_rng(7)
    L = rng.normal(size=oracle.NMI)
    t = np.array([0.011, -0.007, 0.004])
    u = np.array([0.003, 0.002, -0.005])
    a1, p1 = oracle.l2p(oracle.l2l(L, t), u)
    a2, p2 = oracle.l2p(L, t + u)
    assert np.allclose(a1, a2, rtol=1e-12, atol=1e-15)
    assert p1 == pytest.approx(p2, rel=1e-12)


def test_p2l_and_m2l_converge_to_direct():
    rng = np.random.default_rng(9)
    k = 30
    src = 0.5 + 0.01 * (rng.random((3, k)) - 0.5)
    m = rng.random(k)
    z = (src * m).sum(axis=1) / m.sum()
    M = oracle.p2m(src, m, z)
    eps2 = 1e-6
    c = z + np.array([0.12, -0.09, 0.05])
    u = np.array([0.004, 0.003, -0.002])
    L = oracle.m2l(M, z, c, eps2)
    Lp = sum(oracle.p2l(m[j], src[:, j], c, eps2) for j in range(k))
    ref, rp = oracle.direct(np.concatenate([src, (c + u)[:, None]], axis=1), np.append(m, 0.0), 1e-3, [k])
    for LL, tol in ((L, 1e-6), (Lp, 1e-6)):
        acc, pot = oracle.l2p(LL, u)
        assert np.linalg.norm(acc - ref[:, 0]) < tol * np.linalg.norm(ref[:, 0])
        assert abs(pot - rp[0]) < tol * abs(rp[0])
    # a single particle's local expansion at its own centre is exactly the pair force
    L1 = oracle.p2l(m[0], src[:, 0], c, eps2)
    acc, pot = oracle.l2p(L1, np.zeros(3))
    ref1, rp1 = oracle.direct(np.stack([src[:, 0], c], axis=1), np.array([m[0], 0.0]), 1e-3, [1])
    assert np.allclose(acc, ref1[:, 0], rtol=1e-13)
    assert pot == pytest.approx(rp1[0], rel=1e-13)


def test_l2p_error_grows_as_fifth_power_of_the_offset():
    """A local expansion to order 5 is the Taylor polynomial of degree 5 of the far field about
    its centre: the potential's remainder is of order 6 in the offset u, so the force error grows
    as |u|^5 (the expected slope is 5, the next term's order)."""
    c = np.array([0.5, 0.5, 0.5])
    src = c + np.array([0.31, -0.22, 0.27])
    m = 0.8
    L = oracle.p2l(m, src, c, 0.0)
    dirn = np.array([0.36, 0.48, -0.8])
    rs = np.array([0.02, 0.04, 0.08])
    errs = []
    for r in rs:
        acc, _ = oracle.l2p(L, r * dirn)
        ref, _ = oracle.direct(np.stack([src, c + r * dirn], axis=1), np.array([m, 0.0]), 0.0, [1])
        errs.append(np.linalg.norm(acc - ref[:, 0]) / np.linalg.norm(ref[:, 0]))
    slope = np.polyfit(np.log(rs), np.log(errs), 1)[0]
    assert 4.8 < slope < 6.2, slope


def test_plummer_sphere_far_field_is_a_point_mass():
    """Far outside a Plummer sphere of scale a the field tends to M / r^2 along the radius; the
    sampled sphere's residual quadrupole falls off as (a / r)^2 relative."""
    rng = np.random.default_rng(31)
    n, a = 4000, 0.01
    r = a / np.sqrt(rng.random(n) ** (-2.0 / 3.0) - 1.0)
    r = np.minimum(r, 0.2)
    cz = 2.0 * rng.random(n) - 1.0
    ph = 2.0 * np.pi * rng.random(n)
    sz = np.sqrt(1.0 - cz * cz)
    c = np.array([0.3, 0.3, 0.3])
    pos = c[:, None] + r * np.stack([sz * np.cos(ph), sz * np.sin(ph), cz])
    mass = np.full(n, 1.0 / n)
    probe = c + 0.6 * np.array([0.6, 0.64, 0.48])
    ref, _ = oracle.direct(np.concatenate([pos, probe[:, None]], axis=1), np.append(mass, 0.0), 0.0, [n])
    d = probe - (pos * mass).sum(axis=1) / mass.sum()
    point = -mass.sum() * d / np.linalg.norm(d) ** 3
    assert np.linalg.norm(ref[:, 0] - point) <= 1e-3 * np.linalg.norm(point)


# ---------------------------------------------------------------- plain FMM


def _rel_err(a, ref):
    return np.linalg.norm(a - ref, axis=0) / np.linalg.norm(ref, axis=0)


def test_fmm_theta_to_zero_is_direct_sum():
    pos, mass = synth.clustered_plummer(2048, 21)
    ref, rp = oracle.direct(pos, mass, 1e-3)
    f = oracle.FMM(pos, mass, 1e-3, 1e-5)
    acc, pot = f.forces()
    assert _rel_err(acc, ref).max() < 1e-11
    assert np.abs(pot - rp).max() < 1e-11 * np.abs(rp).max()
    assert f.counts()["pc_pairs"] == 0


def test_fmm_accuracy_and_monotone_in_theta():
    pos, mass = synth.clustered_plummer(4096, 1)
    ref, _ = oracle.direct(pos, mass, 1e-3)
    rms = []
    for th in (0.4, 0.55, 0.7, 0.9):
        acc, _ = oracle.FMM(pos, mass, 1e-3, th).forces()
        e = _rel_err(acc, ref)
        rms.append(math.sqrt(np.mean(e ** 2)))
    assert all(a < b for a, b in zip(rms, rms[1:]))
    assert rms[1] < 1e-4  # theta = 0.55
    assert rms[2] < 1e-3  # theta = 0.7


def test_fmm_tree_invariants():
    pos, mass = synth.clustered_plummer(3000, 4)
    pos[:, :40] = pos[:, 40:41]  # a pile of coincident points -> identical keys
    f = oracle.FMM(pos, mass, 1e-3, 0.7)
    keys = f.keys()
    perm = f.perm()
    assert np.all(np.diff(keys.astype(np.float64)) >= 0)
    # stable: equal keys keep the input order
    same = keys[1:] == keys[:-1]
    assert np.all(perm[1:][same] > perm[:-1][same])
    assert sorted(perm.tolist()) == list(range(3000))
    cl = f.cells()
    first, count, child = cl["first"], cl["count"], cl["child"]
    leaves = child[:, 0] < 0
    assert np.all(count[leaves] <= 16) and np.all(count[~leaves] > 16)
    order = np.argsort(first[leaves])
    lf, lc = first[leaves][order], count[leaves][order]
    assert lf[0] == 0 and np.all(lf[1:] == (lf + lc)[:-1]) and (lf + lc)[-1] == 3000
    inner = np.where(~leaves)[0]
    c0, c1 = child[inner, 0], child[inner, 1]
    assert np.all(first[c0] == first[inner]) and np.all(first[c1] == first[c0] + count[c0])
    assert np.all(count[c0] + count[c1] == count[inner])
    assert np.allclose(cl["mass"][c0] + cl["mass"][c1], cl["mass"][inner], rtol=1e-12)
    com = cl["com"]
    mc = (cl["mass"][c0, None] * com[c0] + cl["mass"][c1, None] * com[c1]) / cl["mass"][inner, None]
    assert np.allclose(mc, com[inner], rtol=1e-12, atol=1e-14)
    # bounding boxes and b_max by brute force
    sp = pos[:, perm]
    for c in range(len(first)):
        p = sp[:, first[c]:first[c] + count[c]]
        assert np.all(p.min(axis=1) == cl["lo"][c]) and np.all(p.max(axis=1) == cl["hi"][c])
        d = np.sqrt(((p - com[c][:, None]) ** 2).sum(axis=0)).max()
        assert cl["bmax"][c] == pytest.approx(d, rel=1e-12, abs=1e-300)


@pytest.mark.parametrize("theta", [0.4, 0.7])
def test_fmm_lists_satisfy_the_opening_rule(theta, paper):
    """Every list entry against the rule that produced it (Sec. 3.1, R4), re-checked in FP64 from
    the tree's own geometry: CC/CP entries pass the acceptance test; PC entries fail it and have
    every sink particle outside the source's opening sphere; PP entries fail both (or are
    point-like sources).  Decisions are taken in FP32, so comparisons allow a relative 1e-5.
    The factor of the sink's radius and the gap in softenings are the paper's printed values."""
    pos, mass = synth.clustered_plummer(3000, 15)
    eps, b, g = 1e-3, 16, 64
    fk, fgap = paper["sink_radius_factor"], paper["bbox_gap_softenings"]
    f = oracle.FMM(pos, mass, eps, theta, bucket=b, group=g)
    cl = f.cells()
    first, count, com, lo, hi, bmax = cl["first"], cl["count"], cl["com"], cl["lo"], cl["hi"], cl["bmax"]
    cell_of = {(int(a), int(c)): i for i, (a, c) in enumerate(zip(first, count))}
    ro = np.where(count == 1, 0.0, bmax / theta)
    sp = pos[:, f.perm()]
    tol = 1e-5

    def source(fi, ci):
        """(centre, lo, hi, R_O, b_max, point-like) of an entry's source: a cell, or one particle."""
        c = cell_of.get((fi, ci)) if ci > 1 or (fi, ci) in cell_of else None
        if ci == 1:
            x = sp[:, fi]
            return x, x, x, 0.0, 0.0, True
        return com[c], lo[c], hi[c], ro[c], bmax[c], False

    def accepted(k, src):
        x, slo, shi, sro, _, _ = src
        d = np.linalg.norm(com[k] - x)
        gap = np.linalg.norm(np.maximum(np.maximum(slo - hi[k], lo[k] - shi), 0.0))
        return d, gap, d > (fk * ro[k] + sro) * (1 - tol) and gap >= fgap * eps * (1 - tol), \
            d <= (fk * ro[k] + sro) * (1 + tol) or gap < fgap * eps * (1 + tol)

    for kind in ("cc", "cp"):
        sink, fi, ci = f.entries(kind)
        for k, a, c in zip(sink, fi, ci):
            _, _, ok, _ = accepted(k, source(int(a), int(c)))
            assert ok, (kind, k, a, c)
    for kind in ("pc", "pp"):
        sink, fi, ci = f.entries(kind)
        for k, a, c in zip(sink, fi, ci):
            assert count[k] <= g  # interactions are listed at groups only
            src = source(int(a), int(c))
            d, _, _, rejected = accepted(k, src)
            assert rejected, (kind, k, a, c)
            outside = d > (src[3] + bmax[k]) * (1 - tol)
            if kind == "pc":
                assert not src[5] and outside, (k, a, c)
            else:
                # a particle, or a bucket too close for PC
                assert src[5] or (c <= b and d <= (src[3] + bmax[k]) * (1 + tol)), (k, a, c)


def test_fmm_group_locals_are_the_sum_of_their_accepted_sources():
    """A group's local expansion is every CC/CP entry of the group and of its ancestors, each
    expanded about the centre of mass of the cell that accepted it and shifted to the group's
    (L2L is exact on the degree-5 polynomial).  Rebuilt here from the exported lists and tree."""
    pos, mass = synth.clustered_plummer(2000, 16)
    eps = 1e-3
    f = oracle.FMM(pos, mass, eps, 0.6, bucket=8, group=32)
    cl = f.cells()
    first, count, parent, com = cl["first"], cl["count"], cl["parent"], cl["com"]
    cell_of = {(int(a), int(c)): i for i, (a, c) in enumerate(zip(first, count))}
    sp, sm = pos[:, f.perm()], mass[f.perm()]
    own = {}
    for kind in ("cc", "cp"):
        sink, fi, ci = f.entries(kind)
        for k, a, c in zip(sink, fi, ci):
            if c == 1:
                L = oracle.p2l(sm[a], sp[:, a], com[k], eps * eps)
            else:
                s_ = cell_of[(int(a), int(c))]
                L = oracle.m2l(cl["mom"][s_], com[s_], com[k], eps * eps)
            own[int(k)] = own.get(int(k), 0.0) + L
    gcell, gL = f.groups()
    assert len(own) > 10
    for g, Lg in zip(gcell[::7], gL[::7]):
        want = np.zeros(oracle.NMI)
        k = int(g)
        while k >= 0:
            if k in own:
                want += oracle.l2l(own[k], com[g] - com[k])
            k = int(parent[k])
        assert np.allclose(Lg, want, rtol=1e-10, atol=1e-10 * np.max(np.abs(want))), g


def test_fmm_morton_keys_known_points():
    """Level l bisects axis l mod 3 (x, y, z): the key's top three bits are x, y, z halves."""
    pos = np.array([[0.75, 0.25, 0.25, 0.25, 0.0], [0.25, 0.75, 0.25, 0.25, 0.0], [0.25, 0.25, 0.75, 0.25, 0.0]])
    f = oracle.FMM(pos, np.ones(5) / 5, 1e-3, 0.7)
    k = dict(zip(f.perm().tolist(), f.keys().tolist()))
    assert k[4] == 0
    assert k[0] >> 60 == 0b100 and k[1] >> 60 == 0b010 and k[2] >> 60 == 0b001 and k[3] >> 60 == 0
    # 0.25 = 0.01b in every axis: level-3..5 bits are all one
    assert (k[3] >> 57) & 0b111 == 0b111


def _coverage(f, n):
    """For every active sink particle, the number of source particles reached through PP, PC and
    the CC/CP lists of the sink's group and all its ancestors."""
    cl = f.cells()
    first, count, parent = cl["first"], cl["count"], cl["parent"]
    per_cell = np.zeros(len(first), np.int64)
    for kind in ("cc", "cp"):
        s, _, c = f.entries(kind)
        np.add.at(per_cell, s, c)
    gcell, _ = f.groups()
    tot = {}
    for kind in ("pp", "pc"):
        s, _, c = f.entries(kind)
        for si, ci in zip(s, c):
            tot[si] = tot.get(si, 0) + ci
    out = []
    for g in gcell:
        t = tot.get(g, 0)
        a = g
        while a >= 0:
            t += per_cell[a]
            a = parent[a]
        out.append((g, t))
    return out


@pytest.mark.parametrize("theta", [0.4, 0.7, 1.0])
def test_fmm_walk_covers_every_source_exactly_once(theta):
    pos, mass = synth.clustered_plummer(2500, 8)
    f = oracle.FMM(pos, mass, 1e-3, theta)
    cov = _coverage(f, 2500)
    assert len(cov) > 10
    assert all(t == 2500 for _, t in cov)


def test_fmm_active_subset_matches_full_solve():
    pos, mass = synth.clustered_plummer(3000, 12)
    act = (np.arange(3000) % 7 == 0).astype(np.uint8)
    full, fp = oracle.FMM(pos, mass, 1e-3, 0.7).forces()
    part, pp = oracle.FMM(pos, mass, 1e-3, 0.7, active=act).forces(fill=np.nan)
    sel = act.astype(bool)
    assert np.array_equal(part[:, sel], full[:, sel]) and np.array_equal(pp[sel], fp[sel])
    assert np.all(np.isnan(part[:, ~sel]))


def test_fmm_tiny_n_and_degenerate_sets():
    for n in (1, 2, 3, 17, 64, 65):
        pos, mass = synth.clustered_plummer(n, 30 + n)
        acc, pot = oracle.FMM(pos, mass, 1e-3, 0.7).forces()
        ref, rp = oracle.direct(pos, mass, 1e-3)
        assert _rel_err(acc, ref).max() < 1e-3 if n > 1 else np.all(acc == 0)
    # coincident points: identical keys split by position, b_max = 0 cells.  The local
    # expansion of a sink cell spanning two points is still truncated at r/d < theta/1.5,
    # so the error bound is (theta/1.5)^5 ~ 3e-4 at theta = 0.3.
    pos, mass = synth.coincident(200, 3, n_points=3)
    f = oracle.FMM(pos, mass, 1e-3, 0.3)
    acc, pot = f.forces()
    ref, rp = oracle.direct(pos, mass, 1e-3)
    assert _rel_err(acc, ref).max() < 1e-3
    assert all(t == 200 for _, t in _coverage(f, 200))
