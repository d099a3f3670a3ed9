"""Dual trees for multiple time steps (Sec. 3.2), through the C ABI.

The particles of the slow rungs (rung <= r_fixed) are drifted to the middle of their interval,
x + v dt, and kept in a fixed tree. Each substep builds a tree of every other particle at its
current position and walks the sinks (the particles active on the substep) against both trees.
What the method approximates is the direct sum over the union of the two sets.
So each solve is checked against the oracle's FP64 direct sum of that union, to the method's
accuracy target (rms <= 1e-3, 99th percentile <= 1e-2). Exact checks pin the compaction, the
relabelling of the appended tree and the output order: an empty fixed set reproduces a plain
solve bit for bit.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1609_08621_gb300 import binding, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = binding.Context(0, bucket=16, group=64)
    yield c
    c.close()


def _t(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a).reshape(-1)).to("cuda:0", dtype)


def _rel_err(a, ref):
    return np.linalg.norm(a - ref, axis=0) / np.linalg.norm(ref, axis=0)


def _assert_accuracy(e):
    rms = float(np.sqrt(np.mean(np.square(e))))
    assert rms <= 1e-3 and float(np.quantile(e, 0.99)) <= 1e-2, (rms, float(np.quantile(e, 0.99)))


def _particles(n, seed, dt):
    """Clustered positions, rungs 0..5 and velocities whose drift over dt stays in the box."""
    pos, mass = synth.clustered_plummer(n, seed)
    rng = np.random.default_rng(seed)
    rung = rng.integers(0, 6, n).astype(np.uint8)
    target = np.clip(pos + rng.normal(0.0, 2e-3, pos.shape), 1e-6, 1.0 - 1e-6)
    vel = (target - pos) / dt
    return pos, mass, rung, vel


def _union(pos, vel, dt, fixed):
    """The drifted positions of the fixed particles, computed as the library does (x + v dt,
    each operation rounded)."""
    u = pos.copy()
    u[:, fixed] = pos[:, fixed] + vel[:, fixed] * dt
    return u


def _solve_dual(ctx, pos, mass, rung, vel, dt, r_fixed, active, eps, theta):
    n = mass.size
    tp, tm = _t(pos, torch.float64), _t(mass, torch.float32)
    ctx.set_fixed_sources(tp, tm, _t(rung, torch.uint8), r_fixed, _t(vel, torch.float64), dt)
    acc = torch.full((3 * n,), float("nan"), dtype=torch.float32, device="cuda:0")
    pot = torch.full((n,), float("nan"), dtype=torch.float32, device="cuda:0")
    ctx.compute_forces_dual(tp, tm, eps, theta, acc, pot, _t(active, torch.uint8))
    return acc.cpu().numpy().reshape(3, n).astype(np.float64), pot.cpu().numpy().astype(np.float64)


def test_dual_solve_matches_direct_sum_of_the_union(ctx):
    n, eps, theta, dt = 20000, 1e-3, 0.6, 0.5
    pos, mass, rung, vel = _particles(n, 21, dt)
    fixed = rung <= 3
    active = (~fixed).astype(np.uint8)
    a, p = _solve_dual(ctx, pos, mass, rung, vel, dt, 3, active, eps, theta)
    act = active.astype(bool)
    assert np.all(np.isnan(a[:, ~act])) and np.all(np.isnan(p[~act]))
    assert np.all(np.isfinite(a[:, act]))
    st = ctx.stats()
    assert st["n_pp_pairs"] > 0 and st["n_pc_pairs"] > 0
    u = _union(pos, vel, dt, fixed)
    sinks = np.flatnonzero(act)
    ref, rp = oracle.direct(u, mass, eps, sinks)
    _assert_accuracy(_rel_err(a[:, sinks], ref))
    assert float(np.sqrt(np.mean(((p[sinks] - rp) / rp) ** 2))) <= 1e-3
    # the single-tree solve of the same union approximates the same sum
    tacc = torch.zeros(3 * n, dtype=torch.float32, device="cuda:0")
    ctx.compute_forces(_t(u, torch.float64), _t(mass, torch.float32), eps, theta, tacc, None, _t(active, torch.uint8))
    a1 = tacc.cpu().numpy().reshape(3, n).astype(np.float64)
    _assert_accuracy(_rel_err(a[:, sinks], a1[:, sinks]))


def test_empty_fixed_set_is_a_plain_solve(ctx):
    """With no fixed particle every particle is in the active tree, so the dual solve is the
    plain solve of the same sinks: the same tree, lists and sums, written in the same places."""
    n, eps, theta, dt = 12000, 1e-3, 0.6, 0.5
    pos, mass, rung, vel = _particles(n, 22, dt)
    active = (rung >= 2).astype(np.uint8)
    a, p = _solve_dual(ctx, pos, mass, rung, vel, dt, -1, active, eps, theta)  # no rung <= -1
    acc = torch.full((3 * n,), float("nan"), dtype=torch.float32, device="cuda:0")
    pot = torch.full((n,), float("nan"), dtype=torch.float32, device="cuda:0")
    ctx.compute_forces(_t(pos, torch.float64), _t(mass, torch.float32), eps, theta, acc, pot, _t(active, torch.uint8))
    assert np.array_equal(a, acc.cpu().numpy().reshape(3, n).astype(np.float64), equal_nan=True)
    assert np.array_equal(p, pot.cpu().numpy().astype(np.float64), equal_nan=True)


def test_one_fixed_tree_serves_several_active_sets(ctx):
    n, eps, theta, dt = 16000, 1e-3, 0.6, 0.25
    pos, mass, rung, vel = _particles(n, 23, dt)
    fixed = rung <= 2
    tp, tm = _t(pos, torch.float64), _t(mass, torch.float32)
    ctx.set_fixed_sources(tp, tm, _t(rung, torch.uint8), 2, _t(vel, torch.float64), dt)
    u_fixed = _union(pos, vel, dt, fixed)
    rng = np.random.default_rng(5)
    for step in range(2):
        # the active particles move between solves; the fixed tree stays
        cur = pos.copy()
        mov = ~fixed
        cur[:, mov] = np.clip(pos[:, mov] + rng.normal(0.0, 1e-3, (3, int(mov.sum()))), 1e-6, 1 - 1e-6)
        active = np.zeros(n, np.uint8)
        active[mov] = 1
        if step == 1:
            active[np.flatnonzero(mov)[::2]] = 0  # a subset of the fast rungs
        acc = torch.full((3 * n,), float("nan"), dtype=torch.float32, device="cuda:0")
        ctx.compute_forces_dual(_t(cur, torch.float64), tm, eps, theta, acc, None, _t(active, torch.uint8))
        a = acc.cpu().numpy().reshape(3, n).astype(np.float64)
        u = cur.copy()
        u[:, fixed] = u_fixed[:, fixed]
        # sources: every particle (the fast rungs, active or not, in the active tree); sinks: the
        # active ones
        sinks = np.flatnonzero(active)
        ref, _ = oracle.direct(u, mass, eps, sinks)
        _assert_accuracy(_rel_err(a[:, sinks], ref))
        assert np.all(np.isnan(a[:, active == 0]))


def test_errors_and_empty_active_set():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    n = 3000
    pos, mass, rung, vel = _particles(n, 24, 1.0)
    tp, tm = _t(pos, torch.float64), _t(mass, torch.float32)
    acc = torch.full((3 * n,), float("nan"), dtype=torch.float32, device="cuda:0")
    c = binding.Context(0, bucket=16, group=64)
    try:
        with pytest.raises(binding.FmmError) as e:  # no fixed tree yet
            c.compute_forces_dual(tp, tm, 1e-3, 0.6, acc)
        assert e.value.status == binding.FMM_ERR_STATE
        c.set_fixed_sources(tp, tm, _t(rung, torch.uint8), 1)
        c.set_params(bucket=12)
        with pytest.raises(binding.FmmError) as e:  # bucket differs from the fixed tree's
            c.compute_forces_dual(tp, tm, 1e-3, 0.6, acc)
        assert e.value.status == binding.FMM_ERR_ARG
        c.set_params(bucket=16)
        with pytest.raises(binding.FmmError) as e:  # not the particle set the fixed set came from
            c.compute_forces_dual(tp[: 3 * (n - 1)], tm[: n - 1], 1e-3, 0.6, acc[: 3 * (n - 1)])
        assert e.value.status == binding.FMM_ERR_ARG
        with pytest.raises(binding.FmmError):
            c.set_fixed_sources(tp, tm, None, 0, _t(vel, torch.float64), float("inf"))
        c.set_fixed_sources(tp, tm, _t(rung, torch.uint8), 1)
        c.compute_forces_dual(tp, tm, 1e-3, 0.6, acc, None, torch.zeros(n, dtype=torch.uint8, device="cuda:0"))
        assert bool(torch.isnan(acc).all())  # no active particle: nothing written
    finally:
        c.close()


def test_full_size_256cubed_fast_rungs(ctx):
    """The 256^3 box, fixed rungs <= 3 at their interval's middle, the fast rungs active: sampled
    sinks against the FP64 direct sum of the union."""
    n = 256 ** 3
    eps, theta, dt = synth.paper_softening(n), 0.55, 0.5
    pos, mass = synth.clustered_plummer(n, 4)
    rng = np.random.default_rng(25)
    rung = rng.choice(np.arange(6, dtype=np.uint8), n, p=[0.0, 0.01, 0.47, 0.08, 0.34, 0.10])
    target = np.clip(pos + rng.normal(0.0, 1e-4, pos.shape), 1e-6, 1.0 - 1e-6)
    vel = (target - pos) / dt
    fixed = rung <= 3
    active = (~fixed).astype(np.uint8)
    a, _ = _solve_dual(ctx, pos, mass, rung, vel, dt, 3, active, eps, theta)
    u = _union(pos, vel, dt, fixed)
    sinks = rng.choice(np.flatnonzero(active), 256, replace=False)
    ref, _ = oracle.direct(u, mass, eps, sinks)
    _assert_accuracy(_rel_err(a[:, sinks], ref))


@pytest.mark.parametrize("n", [2, 3, 17, 100])
def test_tiny_sets(ctx, n):
    """Trees of one or a few particles on either side: the solve is still the direct sum of the
    union (almost all of it PP at these sizes)."""
    dt = 0.5
    pos, mass, rung, vel = _particles(n, 40 + n, dt)
    rung[0], rung[1] = 5, 0  # at least one fast and one fixed particle
    fixed = rung <= 2
    active = (~fixed).astype(np.uint8)
    a, p = _solve_dual(ctx, pos, mass, rung, vel, dt, 2, active, 1e-3, 0.6)
    assert np.all(np.isnan(a[:, fixed]))
    sinks = np.flatnonzero(active)
    ref, _ = oracle.direct(_union(pos, vel, dt, fixed), mass, 1e-3, sinks)
    assert _rel_err(a[:, sinks], ref).max() <= 2e-3


def test_everything_fixed_writes_nothing(ctx):
    n = 500
    pos, mass, _, _ = _particles(n, 26, 1.0)
    tp, tm = _t(pos, torch.float64), _t(mass, torch.float32)
    ctx.set_fixed_sources(tp, tm)  # no rungs: every particle is fixed
    acc = torch.full((3 * n,), float("nan"), dtype=torch.float32, device="cuda:0")
    ctx.compute_forces_dual(tp, tm, 1e-3, 0.6, acc)
    assert bool(torch.isnan(acc).all())
