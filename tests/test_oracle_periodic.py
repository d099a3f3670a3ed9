"""Pins of the periodic oracle (Sec. 3.1: the root and its 26 or 124 replicas on the checklist, the
copies beyond from a 5th-order multipole approximation of the Ewald sum).

The periodic direct sum is pinned by what the lattice fixes independently of the Ewald formulas:
- the Wigner constant of the simple cubic lattice;
- the r^2 term of the periodic potential;
- the symmetries of a sub-lattice and of a body-centred pair;
- independence of the Ewald split parameter;
- -grad of the potential, momentum and translation invariance;
- the limit of a compact cluster in a large box.

The correction kernel's derivatives are pinned by finite differences, Laplace's equation with the
background (nabla^2 F = 4 pi, higher traces zero), split independence and cubic symmetry. The
periodic FMM is pinned by brute force over the copies, exact coverage of every (source, copy)
pair, and its accuracy against the periodic direct sum.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1609_08621_gb300 import synth

MI = oracle.multi_index()
IDX = {tuple(int(v) for v in row): i for i, row in enumerate(MI)}

# Wigner constant of the simple cubic lattice (Madelung-type sum of a point charge on the lattice
# of unit spacing with a neutralising background): the regular part of the periodic potential at
# the origin, lim_{r->0} psi(r) - 1/r.
XI_SC = -2.837297479480620


def _rel_err(a, ref):
    return np.linalg.norm(a - ref, axis=0) / np.linalg.norm(ref, axis=0)


# ---------------------------------------------------------------- periodic direct sum


@pytest.mark.parametrize("nrep", [1, 2])
@pytest.mark.parametrize("alpha", [3.0, 5.0, 8.0])
def test_lone_particle_sees_the_wigner_constant(nrep, alpha):
    """A single particle interacts only with its own copies and the background: no force, and the
    potential -m xi for the simple cubic lattice of unit spacing."""
    pos = np.array([[0.3], [0.4], [0.7]])
    acc, pot = oracle.direct_periodic(pos, np.array([1.7]), 1e-9, nrep=nrep, alpha=alpha)
    assert pot[0] == pytest.approx(-1.7 * XI_SC, rel=1e-12)
    assert np.all(np.abs(acc) < 1e-12)


def test_sub_lattice_scales_the_wigner_constant():
    """Eight equal masses on the lattice of spacing 1/2 form the simple cubic lattice of that
    spacing, whose potential at a site is -m xi / a = -2 m xi; by symmetry no site feels a force."""
    rng = np.random.default_rng(1)
    off = rng.random(3) * 0.5
    g = np.array([[i, j, k] for i in (0, 0.5) for j in (0, 0.5) for k in (0, 0.5)]).T
    pos = (g + off[:, None]) % 1.0
    m = np.full(8, 0.3)
    acc, pot = oracle.direct_periodic(pos, m, 1e-9)
    assert np.allclose(pot, -2.0 * 0.3 * XI_SC, rtol=1e-12)
    assert np.all(np.abs(acc) < 1e-11)


def test_body_centred_pair_feels_no_force():
    pos = np.array([[0.1, 0.6], [0.2, 0.7], [0.3, 0.8]])
    acc, pot = oracle.direct_periodic(pos, np.array([1.0, 2.5]), 1e-9)
    assert np.all(np.abs(acc) < 1e-11)
    # both sites of the body-centred lattice: pot_i = -m_i xi - m_other psi((1/2,1/2,1/2))
    assert pot[0] + 1.0 * XI_SC == pytest.approx((pot[1] + 2.5 * XI_SC) * 2.5, rel=1e-12)


def test_close_pair_is_newton_plus_the_background_term():
    """psi(r) = 1/r + xi + (2 pi / 3) r^2 + O(r^4): a close pair feels Newton's force plus the
    background's (4 pi / 3) m r, and the potential follows the expansion."""
    d = 0.01
    u = np.array([0.6, -0.48, 0.64])
    u /= np.linalg.norm(u)
    x1 = np.array([0.5, 0.5, 0.5])
    x2 = x1 + d * u
    m = np.array([1.0, 2.0])
    acc, pot = oracle.direct_periodic(np.stack([x1, x2], 1), m, 1e-9)
    r = x1 - x2
    extra = acc[:, 0] - m[1] * (-r) / d ** 3
    assert np.allclose(extra, 4.0 * math.pi / 3.0 * m[1] * r, rtol=1e-3)
    expect = -m[1] * (1.0 / d + XI_SC + 2.0 * math.pi / 3.0 * d * d) - m[0] * XI_SC
    assert pot[0] == pytest.approx(expect, rel=1e-9)


def test_split_parameter_and_shell_independence():
    """The Ewald split parameter changes nothing.  The size of the shell only moves the line
    between softened and Newtonian copies, which at eps = 1e-3 changes forces by O(eps^2)."""
    pos, m = synth.clustered_plummer(300, 7)
    a3, p3 = oracle.direct_periodic(pos, m, 1e-3, alpha=3.0)
    a8, p8 = oracle.direct_periodic(pos, m, 1e-3, alpha=8.0)
    assert np.max(_rel_err(a3, a8)) < 1e-11
    assert np.allclose(p3, p8, rtol=1e-12)
    # each source's softened and Newtonian pulls at distance >= 1/2 differ by < (3/2) eps^2 / r^4
    a2, p2 = oracle.direct_periodic(pos, m, 1e-3, nrep=2)
    assert np.max(np.linalg.norm(a2 - a8, axis=0)) < 30 * 1e-6 * m.sum()
    assert np.max(np.abs(p2 - p8)) < 10 * 1e-6 * m.sum()


def test_periodic_force_is_minus_gradient_and_momentum_vanishes():
    rng = np.random.default_rng(2)
    n = 6
    pos = rng.random((3, n))
    m = 0.5 + rng.random(n)
    eps = 0.02
    acc, _ = oracle.direct_periodic(pos, m, eps)
    # moving particle i (and its copies): a_i = -d phi_i / d x_i
    h = 1e-5
    for i in range(n):
        for a in range(3):
            pp, pm = pos.copy(), pos.copy()
            pp[a, i] += h
            pm[a, i] -= h
            fd = -(oracle.direct_periodic(pp, m, eps, [i])[1][0] - oracle.direct_periodic(pm, m, eps, [i])[1][0])
            assert fd / (2 * h) == pytest.approx(acc[a, i], rel=1e-6, abs=1e-6)
    mom = (m * acc).sum(axis=1)
    assert np.all(np.abs(mom) < 1e-12 * (m * np.abs(acc)).sum())


def test_translation_modulo_the_box():
    """Shifting every particle by a vector and wrapping into the box changes nothing (up to which
    copies are softened: O(eps^2))."""
    pos, m = synth.clustered_plummer(200, 8)
    acc, pot = oracle.direct_periodic(pos, m, 1e-3)
    moved = (pos + np.array([[0.37], [0.81], [0.45]])) % 1.0
    acc2, pot2 = oracle.direct_periodic(moved, m, 1e-3)
    assert np.max(np.linalg.norm(acc2 - acc, axis=0)) < 30 * 1e-6 * m.sum()
    assert np.max(np.abs(pot2 - pot)) < 10 * 1e-6 * m.sum()


def test_compact_cluster_in_a_large_box():
    """A cluster much smaller than the box feels its own isolated field plus the background's
    linear term (4 pi / 3) M (x - x_com); the copies' tidal field enters at the next order."""
    rng = np.random.default_rng(3)
    n = 200
    pos = 0.5 + 0.01 * rng.normal(size=(3, n))
    m = rng.random(n) / n
    per, _ = oracle.direct_periodic(pos, m, 1e-4)
    iso, _ = oracle.direct(pos, m, 1e-4)
    com = (pos * m).sum(axis=1, keepdims=True) / m.sum()
    lin = 4.0 * math.pi / 3.0 * m.sum() * (pos - com)
    assert np.max(np.linalg.norm(per - iso - lin, axis=0) / np.linalg.norm(lin, axis=0)) < 1e-2


# ---------------------------------------------------------------- Ewald correction kernel


def test_ewald_derivs_against_finite_differences():
    h = 1e-5
    for r0 in (np.array([0.31, -0.47, 0.22]), np.array([-0.85, 0.6, 0.9]), np.zeros(3)):
        D = oracle.ewald_derivs(r0)
        for i, n in enumerate(MI):
            if n.sum() > 4:
                continue
            for q in range(3):
                e = np.zeros(3)
                e[q] = h
                fd = (oracle.ewald_derivs(r0 + e)[i] - oracle.ewald_derivs(r0 - e)[i]) / (2 * h)
                nn = n.copy()
                nn[q] += 1
                ref = D[IDX[tuple(int(v) for v in nn)]]
                assert fd == pytest.approx(ref, rel=1e-6, abs=1e-5), (r0, n, q)


@pytest.mark.parametrize("nrep", [0, 1, 2])
def test_ewald_kernel_obeys_poisson_with_the_background(nrep):
    """Away from the copies, nabla^2 psi = 4 pi (the background) and every 1/|r+n| is harmonic:
    nabla^2 F = 4 pi and nabla^2 of every higher derivative is zero."""
    for r0 in (np.array([0.31, -0.47, 0.22]), np.array([0.7, 0.05, -0.66])):
        D = oracle.ewald_derivs(r0, nrep=nrep)
        for k in MI:
            if k.sum() > 3:
                continue
            t = sum(D[IDX[tuple(int(v) for v in k + 2 * np.eye(3, dtype=int)[q])]] for q in range(3))
            want = 4.0 * math.pi if k.sum() == 0 else 0.0
            assert t == pytest.approx(want, abs=1e-8 * (1 + np.max(np.abs(D))))


def test_ewald_derivs_independent_of_split_and_cubic_symmetric():
    r0 = np.array([0.31, -0.47, 0.22])
    D = oracle.ewald_derivs(r0, alpha=2.5)
    assert np.allclose(D, oracle.ewald_derivs(r0, alpha=5.5), rtol=1e-10, atol=1e-10)
    # permuting the axes permutes the multi-indices; reflecting x flips the odd-x derivatives
    Dp = oracle.ewald_derivs(r0[[2, 0, 1]])
    Dr = oracle.ewald_derivs(r0 * np.array([-1.0, 1.0, 1.0]))
    for i, (a, b, c) in enumerate(MI):
        assert Dp[IDX[(int(c), int(a), int(b))]] == pytest.approx(D[i], rel=1e-10, abs=1e-10)
        assert Dr[i] == pytest.approx((-1) ** int(a) * D[i], rel=1e-10, abs=1e-10)


def test_shell_plus_correction_is_the_periodic_pair_kernel():
    """The softened copies of the shell plus F, for one source, give the periodic direct sum's pair
    kernel (computed there through structure factors and a pair loop)."""
    rng = np.random.default_rng(4)
    eps = 1e-3
    for _ in range(3):
        pos = rng.random((3, 2))
        m = np.array([0.0, 1.3])  # only the source's field at the sink
        acc, pot = oracle.direct_periodic(pos, m, eps, [0])
        r = pos[:, 0] - pos[:, 1]
        D = oracle.ewald_derivs(r)
        a, p = m[1] * D[1:4], -m[1] * D[0]
        for s in np.ndindex(3, 3, 3):
            u = r + np.array(s) - 1
            R2 = u @ u + eps * eps
            a += -m[1] * u / R2 ** 1.5
            p += -m[1] / math.sqrt(R2)
        assert np.allclose(acc[:, 0], a, rtol=1e-11, atol=1e-11)
        assert pot[0] == pytest.approx(p, rel=1e-12)


def test_ewald_m2p_is_the_moment_expansion_of_the_exact_sum():
    """The 5th-order correction from the moments of a compact set about its centre of mass equals
    sum_j m_j grad F(x - x_j) up to the truncation, which falls as (size / distance)^5."""
    rng = np.random.default_rng(5)
    shape = rng.random((3, 40)) - 0.5
    m = 0.5 + rng.random(40)
    errs = []
    for size in (0.1, 0.05):
        pos = 0.5 + size * shape
        z = (pos * m).sum(axis=1) / m.sum()
        M = oracle.p2m(pos, m, z)
        x = np.array([0.1, 0.85, 0.3])
        a, p = oracle.ewald_m2p(M, z, x)
        ae = np.zeros(3)
        pe = 0.0
        for j in range(40):
            D = oracle.ewald_derivs(x - pos[:, j])
            ae += m[j] * D[1:4]
            pe -= m[j] * D[0]
        errs.append(np.linalg.norm(a - ae) / np.linalg.norm(ae))
        assert p == pytest.approx(pe, rel=1e-6)
    # the same shape at half the size: the first neglected order falls by 2^5
    assert errs[0] < 1e-6 and 24 < errs[0] / errs[1] < 40


# ---------------------------------------------------------------- periodic FMM


def _near_copies(pos, m, eps, sinks, nrep=1):
    """Brute force over the softened copies of the shell (numpy)."""
    acc = np.zeros((3, len(sinks)))
    pot = np.zeros(len(sinks))
    for q, i in enumerate(sinks):
        for s in np.ndindex(*(2 * nrep + 1,) * 3):
            sv = np.array(s)[:, None] - nrep
            d = pos + sv - pos[:, [i]]
            r2 = (d * d).sum(axis=0) + eps * eps
            if not sv.any():
                r2[i] = np.inf
            ir = 1.0 / np.sqrt(r2)
            acc[:, q] += (m * ir ** 3 * d).sum(axis=1)
            pot[q] -= (m * ir).sum()
    return acc, pot


@pytest.mark.parametrize("nrep", [1, 2])
def test_periodic_fmm_tree_part_at_small_theta_is_the_shell_sum(nrep):
    pos, m = synth.clustered_plummer(600, 9)
    eps = 1e-3
    f = oracle.FMM(pos, m, eps, 0.05, nrep=nrep)
    a, p = f.forces(terms=7)
    sinks = np.arange(0, 600, 5)
    an, pn = _near_copies(pos, m, eps, sinks, nrep)
    assert np.max(_rel_err(a[:, sinks], an)) < 1e-7
    assert np.allclose(p[sinks], pn, rtol=1e-8)
    # the Ewald term is the root's moments through the correction kernel
    a8, p8 = f.forces(terms=8)
    cl = f.cells()
    for i in sinks[:10]:
        ae, pe = oracle.ewald_m2p(cl["mom"][0], cl["com"][0], pos[:, i], nrep=nrep)
        assert np.allclose(a8[:, i], ae, rtol=1e-12, atol=1e-12)
        assert p8[i] == pytest.approx(pe, rel=1e-12)


def _copy_coverage(f, n, nrep):
    """count[g, copy, j]: how often source particle j in the given copy reaches the sinks of group
    g, through the group's PP and PC entries and the CC/CP entries of it and its ancestors."""
    cl = f.cells()
    first, count, parent = cl["first"], cl["count"], cl["parent"]
    w = 2 * nrep + 1
    by_cell = {}
    for kind in ("pp", "pc", "cc", "cp"):
        s, fi, c = f.entries(kind)
        sh = f.shifts(kind)
        for si, f0, ci, v in zip(s, fi, c, sh):
            by_cell.setdefault(int(si), []).append((int(f0), int(ci), int(np.ravel_multi_index(v + nrep, (w,) * 3)),
                                                    kind in ("pp", "pc")))
    gcell, _ = f.groups()
    out = []
    for g in gcell:
        cnt = np.zeros((w ** 3, n), np.int64)
        k, own = int(g), True
        while k >= 0:
            for f0, ci, code, near_kind in by_cell.get(k, []):
                if near_kind and not own:
                    continue
                cnt[code, f0:f0 + ci] += 1
            k, own = int(parent[k]), False
        out.append((int(first[g]), int(count[g]), cnt))
    return out


@pytest.mark.parametrize("theta", [0.4, 0.7])
def test_periodic_walk_covers_every_source_copy_exactly_once(theta):
    pos, m = synth.clustered_plummer(1500, 10)
    f = oracle.FMM(pos, m, 1e-3, theta, bucket=8, group=32, nrep=1)
    for f0, c, cnt in _copy_coverage(f, 1500, 1):
        # every (copy, source) once; the sink group's own particles in the box once too (the
        # particle itself is skipped inside PP)
        assert np.all(cnt == 1), (f0, c, np.unique(cnt))


@pytest.mark.parametrize("nrep", [1, 2])
def test_periodic_fmm_meets_the_accuracy_target(nrep):
    """Against the periodic direct sum: rms <= 1e-3 and 99th percentile <= 1e-2 at theta = 0.55;
    the residual at small theta is the 5th-order truncation of the Ewald term."""
    pos, m = synth.clustered_plummer(3000, 11)
    sinks = np.arange(0, 3000, 3)
    ref, rp = oracle.direct_periodic(pos, m, 1e-3, sinks, nrep=nrep)
    f = oracle.FMM(pos, m, 1e-3, 0.55, nrep=nrep)
    a, p = f.forces()
    e = _rel_err(a[:, sinks], ref)
    assert math.sqrt(np.mean(e ** 2)) <= 1e-3 and np.quantile(e, 0.99) <= 1e-2
    assert math.sqrt(np.mean(((p[sinks] - rp) / rp) ** 2)) <= 1e-2


def test_periodic_fmm_rejects_a_shell_out_of_range():
    pos, m = synth.clustered_plummer(50, 12)
    with pytest.raises(ValueError):
        oracle.FMM(pos, m, 1e-3, 0.55, nrep=3)


def test_ewald_correction_is_a_low_degree_polynomial_on_sub_cubes():
    """The correction field of the root's moments is smooth across the box (its nearest singularity
    lies >= 1 outside): on a sub-cube of side 1/4 the best degree-5 polynomial reproduces its force
    to 1e-6 of its size, which is what a grid of order-5 local expansions relies on."""
    import itertools

    pos, m = synth.clustered_plummer(1000, 13)
    z = (pos * m).sum(axis=1) / m.sum()
    M = oracle.p2m(pos, m, z)
    exps = [e for e in itertools.product(range(6), repeat=3) if sum(e) <= 5]
    rng = np.random.default_rng(14)
    h = 0.25
    c = np.array([0.125, 0.125, 0.875])  # a corner sub-cube, the farthest from the centre of mass
    X = c + (rng.random((150, 3)) - 0.5) * h
    acc = np.array([oracle.ewald_m2p(M, z, x)[0] for x in X])
    A = np.array([[np.prod(((x - c) / h) ** np.array(e)) for e in exps] for x in X])
    scale = np.max(np.linalg.norm(acc, axis=1))
    for q in range(3):
        coef, *_ = np.linalg.lstsq(A, acc[:, q], rcond=None)
        assert np.max(np.abs(acc[:, q] - A @ coef)) < 1e-6 * scale
