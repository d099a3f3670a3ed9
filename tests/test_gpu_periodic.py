"""Periodic unit box on the GPU (Sec. 3.1, periodic boundaries: the root and its 26 or 124 copies
on the checklist, the copies beyond from a 5th-order multipole approximation of the Ewald sum;
Sec. 3.3, the Ewald evaluation on the GPU), through the C ABI, against the oracle.

Tolerances:
* interaction lists, with the copy of every source: exact (both sides decide in single precision
  on FP64 geometry shifted in FP64 and then rounded);
* forces term by term against the oracle's periodic FMM on identical lists: the FP32 bounds of the
  isolated box (rms 2e-5, max 2e-3 of |a|); the Ewald term differs from the oracle's per-particle
  evaluation by the Taylor remainder of the correction's order-9 expansions on sub-cubes of side
  1/4, well inside those bounds; potentials relative to the rms of the total potential (in a
  periodic box it has zero mean, so single particles can sit near zero);
* against the oracle's periodic direct sum: the method's accuracy target, rms <= 1e-3 and 99th
  percentile <= 1e-2;
* a lone particle: no force and the potential -m xi of the simple cubic lattice (Wigner constant),
  to the FP32 rounding of the 26 or 124 copy terms and the Ewald grid.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1609_08621_gb300 import binding, synth

pytestmark = pytest.mark.gpu

XI_SC = -2.837297479480620  # Wigner constant of the simple cubic lattice of unit spacing


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = binding.Context(0)
    yield c
    c.close()


def dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a).reshape(-1)).to("cuda:0", dtype)


def solve(ctx, pos, mass, eps, theta, nrep, terms=15, active=None, bucket=16, group=64):
    n = mass.size
    ctx.set_params(terms=terms, nrep=nrep, bucket=bucket, group=group)
    acc = torch.full((3 * n,), float("nan"), dtype=torch.float32, device="cuda:0")
    pot = torch.full((n,), float("nan"), dtype=torch.float32, device="cuda:0")
    act = None if active is None else dev(active, torch.uint8)
    try:
        ctx.compute_forces(dev(pos, torch.float64), dev(mass, torch.float32), eps, theta, acc, pot, act)
        torch.cuda.synchronize()
    finally:
        ctx.set_params(terms=15, nrep=0, bucket=16, group=64)
    return acc.cpu().numpy().reshape(3, n).astype(np.float64), pot.cpu().numpy().astype(np.float64)


def rms(x):
    return float(np.sqrt(np.mean(np.square(x))))


def face_heavy(n, seed):
    """Plummer clusters plus a uniform background, with a tenth of the particles pushed to within
    0.02 of a face or an edge of the box, where the nearest copies are opened down to particles."""
    pos, mass = synth.clustered_plummer(n, seed)
    rng = np.random.default_rng(seed + 100)
    k = n // 10
    idx = rng.choice(n, k, replace=False)
    axis = rng.integers(0, 3, k)
    side = rng.random(k) < 0.5
    pos[axis, idx] = np.where(side, rng.random(k) * 0.02, 1.0 - rng.random(k) * 0.02)
    # corners, edges and faces, including coordinates within 2^-40 of the upper face (their FP32
    # centre rounds to 1, its FP32 low part keeps the offset); no two of them closer than 1e-3 across
    # a face, which FP32 offsets of the group could not resolve
    pos[:, idx[:5]] = np.array([[0.0, 0.0, 0.0], [1.0 - 2.0 ** -40, 0.5, 0.25], [0.0, 0.5, 1.0 - 1e-9],
                                [0.999, 0.001, 0.5], [0.5, 0.0, 0.997]]).T
    return np.ascontiguousarray(pos), mass


def _set_of(rng, sink, first, count, shift):
    return set(zip(map(tuple, rng[sink]), first.tolist(), count.tolist(), map(tuple, shift.tolist())))


@pytest.mark.parametrize("nrep,n,theta", [(1, 6000, 0.55), (1, 5000, 0.7), (2, 2500, 0.55)])
def test_periodic_lists_match_oracle(ctx, nrep, n, theta):
    pos, mass = face_heavy(n, 21 + nrep)
    eps = 1e-3
    solve(ctx, pos, mass, eps, theta, nrep)
    g = ctx.export_cells()
    orc = oracle.FMM(pos, mass, eps, theta, nrep=nrep)
    o = orc.cells()
    grng = np.stack([g["first"], g["count"]], axis=1)
    orng = np.stack([o["first"], o["count"]], axis=1)
    shifted = 0
    for kind in ("pp", "pc", "cc", "cp"):
        s, f, c = ctx.export_lists(kind)
        sh = ctx.export_list_shifts(kind)
        os_, of, oc = orc.entries(kind)
        osh = orc.shifts(kind)
        gs = _set_of(grng, s, f, c, sh)
        ost = _set_of(orng, os_, of, oc, osh)
        assert len(gs) == len(s) and len(ost) == len(os_)
        assert gs == ost, f"{kind}: gpu-only {len(gs - ost)}, oracle-only {len(ost - gs)}"
        shifted += int(np.any(sh != 0, axis=1).sum())
    assert shifted > 0


@pytest.mark.parametrize("nrep", [1, 2])
def test_periodic_forces_match_oracle_fmm_term_by_term(ctx, nrep):
    pos, mass = face_heavy(4000, 31 + nrep)
    eps, theta = 1e-3, 0.55
    orc = oracle.FMM(pos, mass, eps, theta, nrep=nrep)
    tot, totp = orc.forces(15)
    scale = np.linalg.norm(tot, axis=0)
    for terms in (1, 2, 4, 8, 15):
        a, p = solve(ctx, pos, mass, eps, theta, nrep, terms=terms)
        ra, rp = orc.forces(terms)
        e = np.linalg.norm(a - ra, axis=0) / scale
        assert rms(e) <= 2e-5 and e.max() <= 2e-3, (terms, rms(e), e.max())
        ep = np.abs(p - rp) / rms(totp)
        assert rms(ep) <= 2e-5, (terms, rms(ep))


@pytest.mark.parametrize("nrep", [1, 2])
def test_periodic_against_the_periodic_direct_sum(ctx, nrep):
    pos, mass = synth.clustered_plummer(3000, 11)
    eps = 1e-3
    sinks = np.arange(0, 3000, 3)
    ref, rp = oracle.direct_periodic(pos, mass, eps, sinks, nrep=nrep)
    a, p = solve(ctx, pos, mass, eps, 0.55, nrep)
    e = np.linalg.norm(a[:, sinks] - ref, axis=0) / np.linalg.norm(ref, axis=0)
    assert rms(e) <= 1e-3 and np.quantile(e, 0.99) <= 1e-2, (rms(e), np.quantile(e, 0.99))
    assert rms((p[sinks] - rp) / rp) <= 1e-2


@pytest.mark.parametrize("nrep", [1, 2])
def test_lone_particle_sees_the_wigner_constant(ctx, nrep):
    """The particle's own copies in the shell (softened) and the Ewald correction F(0) add up to the
    lattice sum: -m (xi + sum_{0 < |n|_inf <= nrep} (1/sqrt(n^2 + eps^2) - 1/|n|)), with no force.
    eps = 1e-2 keeps the FP32 self term m / eps (170), which the potential sum carries and then
    drops, small: with the copies' terms (|sum| < 110 for nrep 2) every FP32 addition errs by at
    most 2^-24 * 280 = 1.7e-5, and the few dozen additions of a lane's chain stay well below
    4e-5 of the result."""
    pos = np.array([[0.3], [0.4], [0.7]])
    m = np.array([1.7], np.float32)
    eps = 1e-2
    a, p = solve(ctx, pos, m, eps, 0.55, nrep)
    assert np.all(np.abs(a) < 1e-4)
    ns = np.array([v for v in np.ndindex(*(2 * nrep + 1,) * 3)]) - nrep
    n2 = (ns * ns).sum(axis=1).astype(np.float64)
    n2 = n2[n2 > 0]
    expect = -float(m[0]) * (XI_SC + np.sum(1.0 / np.sqrt(n2 + eps * eps) - 1.0 / np.sqrt(n2)))
    assert p[0] == pytest.approx(expect, rel=4e-5)


def test_periodic_64cubed_nfw_active_subset(ctx):
    """A 64^3 NFW box, periodic with nrep = 1, 2048 random active sinks: lists exact and forces at
    FP32 tolerance against the oracle's periodic FMM on the same active subset."""
    n = 64 ** 3
    pos, mass = synth.clustered_nfw(n, 2)
    eps, theta = synth.paper_softening(n), 0.55
    act = np.zeros(n, np.uint8)
    act[np.random.default_rng(5).choice(n, 2048, replace=False)] = 1
    a, p = solve(ctx, pos, mass, eps, theta, 1, active=act)
    orc = oracle.FMM(pos, mass, eps, theta, active=act, nrep=1)
    g = ctx.export_cells()
    o = orc.cells()
    grng = np.stack([g["first"], g["count"]], axis=1)
    orng = np.stack([o["first"], o["count"]], axis=1)
    for kind in ("pp", "pc", "cc", "cp"):
        s, f, c = ctx.export_lists(kind)
        os_, of, oc = orc.entries(kind)
        assert _set_of(grng, s, f, c, ctx.export_list_shifts(kind)) == _set_of(orng, os_, of, oc, orc.shifts(kind))
    ra, rp = orc.forces()
    sel = act.astype(bool)
    e = np.linalg.norm(a[:, sel] - ra[:, sel], axis=0) / np.linalg.norm(ra[:, sel], axis=0)
    assert rms(e) <= 2e-5 and e.max() <= 2e-3, (rms(e), e.max())


def test_periodic_graph_replay_is_bit_identical(ctx):
    pos, mass = face_heavy(20000, 41)
    eps, theta = 1e-3, 0.55
    a0, p0 = solve(ctx, pos, mass, eps, theta, 1)
    ctx.set_graphs(True)
    try:
        outs = [solve(ctx, pos, mass, eps, theta, 1) for _ in range(3)]
        captured, replays = ctx.graph_info()
    finally:
        ctx.set_graphs(False)
    for a, p in outs:
        assert np.array_equal(a, a0) and np.array_equal(p, p0)
    assert captured


def test_periodic_limits(ctx):
    pos, mass = synth.clustered_plummer(1000, 51)
    eps = 1e-3
    t = dev(pos, torch.float64)
    m = dev(mass, torch.float32)
    acc = torch.zeros(3 * 1000, dtype=torch.float32, device="cuda:0")
    # several boxes, the learned criterion, and nrep outside [0, 2] are refused
    ctx.set_params(nrep=1)
    try:
        with pytest.raises(binding.FmmError):
            ctx.compute_forces_batch(t, m, np.array([0, 500, 1000], np.int64), eps, 0.55, acc)
        with pytest.raises(binding.FmmError):
            ctx.set_params(criterion=1)
            ctx.compute_forces(t, m, eps, 0.55, acc)
    finally:
        ctx.set_params(nrep=0, criterion=0)
    with pytest.raises(binding.FmmError):
        ctx.set_params(nrep=3)
    # the context still solves the isolated box afterwards
    ctx.compute_forces(t, m, eps, 0.55, acc)
    torch.cuda.synchronize()
    ref, _ = oracle.direct(pos, mass, eps)
    a = acc.cpu().numpy().reshape(3, 1000).astype(np.float64)
    e = np.linalg.norm(a - ref, axis=0) / np.linalg.norm(ref, axis=0)
    assert rms(e) <= 1e-3
