"""Recovery paths driven from the host, with no GPU fault: the walk's overflow-and-regrow path
(its capacities started small with fmm_debug_walk_capacity) and device allocations that fail
(fmm_debug_fail_allocations), after which the context must stay usable.

Expected results:
* the regrown walk's interaction lists are the oracle's (exact sets), and its forces are bit for
  bit those of a context that never overflowed (the walk is a deterministic function of its input
  once the buffers suffice);
* a failed allocation returns FMM_ERR_OOM; the next calls, hook off, give the same bits as before.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1609_08621_gb300 import binding, synth

pytestmark = pytest.mark.gpu

FMM_ERR_OOM = -2


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def t(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a).reshape(-1)).to("cuda:0", dtype)


def solve(ctx, pos, mass, eps, theta):
    n = mass.size
    acc = torch.zeros(3 * n, dtype=torch.float32, device="cuda:0")
    pot = torch.zeros(n, dtype=torch.float32, device="cuda:0")
    ctx.compute_forces(t(pos, torch.float64), t(mass, torch.float32), eps, theta, acc, pot)
    torch.cuda.synchronize()
    return acc.cpu().numpy(), pot.cpu().numpy()


def _set_of(rng, sink, first, count):
    return set(zip(map(tuple, rng[sink]), first.tolist(), count.tolist()))


@pytest.mark.parametrize("scratch,scale", [(64, 1), (512, 2)])
def test_walk_regrow_gives_the_oracle_lists(dev, scratch, scale):
    n = 20000
    pos, mass = synth.make("nfw", n, 7)
    eps, theta = synth.paper_softening(n), 0.55
    ref_ctx = binding.Context(0)
    small = binding.Context(0)
    try:
        a0, p0 = solve(ref_ctx, pos, mass, eps, theta)
        assert ref_ctx.stats()["retries"] == 0
        small.debug_walk_capacity(scratch, scale)
        a1, p1 = solve(small, pos, mass, eps, theta)
        assert small.stats()["retries"] >= 1
        assert np.array_equal(a0, a1) and np.array_equal(p0, p1)
        g = small.export_cells()
        orc = oracle.FMM(pos, mass, eps, theta)
        o = orc.cells()
        grng = np.stack([g["first"], g["count"]], axis=1)
        orng = np.stack([o["first"], o["count"]], axis=1)
        for kind in ("pp", "pc", "cc", "cp"):
            s, f, c = small.export_lists(kind)
            os_, of, oc = orc.entries(kind)
            assert _set_of(grng, s, f, c) == _set_of(orng, os_, of, oc), kind
        with pytest.raises(binding.FmmError):
            small.debug_walk_capacity(-1, 0)
    finally:
        ref_ctx.close()
        small.close()


@pytest.mark.parametrize("after", [0, 3, 17])
def test_failed_allocation_reports_oom_and_the_context_recovers(dev, after):
    pa, ma = synth.clustered_plummer(2000, 81)
    pb, mb = synth.clustered_plummer(60000, 82)
    eps, theta = 1e-3, 0.7
    ctx = binding.Context(0)
    try:
        a0, p0 = solve(ctx, pa, ma, eps, theta)
        binding.debug_fail_allocations(after)
        try:
            with pytest.raises(binding.FmmError) as ei:
                solve(ctx, pb, mb, eps, theta)  # 30x the particles: the buffers must grow
            assert ei.value.status == FMM_ERR_OOM
        finally:
            binding.debug_fail_allocations(-1)
        # the smaller set again, then the larger one: same bits as a fresh context
        a1, p1 = solve(ctx, pa, ma, eps, theta)
        assert np.array_equal(a0, a1) and np.array_equal(p0, p1)
        b1, q1 = solve(ctx, pb, mb, eps, theta)
        fresh = binding.Context(0)
        try:
            b2, q2 = solve(fresh, pb, mb, eps, theta)
        finally:
            fresh.close()
        assert np.array_equal(b1, b2) and np.array_equal(q1, q2)
    finally:
        binding.debug_fail_allocations(-1)
        ctx.close()


def test_replay_whose_walk_overflows_is_repeated_eagerly(dev):
    """A graph captured while 0.2% of the particles were active holds walk lists sized for them
    (one entry per particle and list, 8192 scratch entries per warp: no regrow for them); with
    every particle active the same replay overflows them (the PP list alone needs 2.3 entries per
    particle).  The kernels after the walk then
    read none of the partly written lists, the solve is repeated eagerly with grown lists, and the
    result is bit for bit that of a context that never overflowed."""
    n = 20000
    pos, mass = synth.make("nfw", n, 93)
    eps, theta = synth.paper_softening(n), 0.55
    few = (np.random.default_rng(3).random(n) < 0.002).astype(np.uint8)
    c = binding.Context(0)
    try:
        c.debug_walk_capacity(8192, 1)
        c.set_graphs(True)
        tp, tm, ta = t(pos, torch.float64), t(mass, torch.float32), t(few, torch.uint8)
        acc = torch.zeros(3 * n, dtype=torch.float32, device="cuda:0")
        pot = torch.zeros(n, dtype=torch.float32, device="cuda:0")
        c.compute_forces(tp, tm, eps, theta, acc, pot, ta)  # eager, then captured
        assert c.graph_info()["captured"] and c.stats()["retries"] == 0
        r0 = c.graph_info()["replays"]
        ta.fill_(1)
        c.compute_forces(tp, tm, eps, theta, acc, pot, ta)  # the replay overflows
        torch.cuda.synchronize()
        assert c.graph_info()["replays"] == r0 and c.stats()["retries"] >= 1
        a1, p1 = acc.cpu().numpy(), pot.cpu().numpy()
        acc.fill_(float("nan"))
        c.compute_forces(tp, tm, eps, theta, acc, pot, ta)  # captured again after the eager repeat
        torch.cuda.synchronize()
        assert c.graph_info()["replays"] == r0 + 1
        assert np.array_equal(acc.cpu().numpy(), a1)
    finally:
        c.close()
    ref = binding.Context(0)
    try:
        a0, p0 = solve(ref, pos, mass, eps, theta)
        assert ref.stats()["retries"] == 0
    finally:
        ref.close()
    assert np.array_equal(a0, a1) and np.array_equal(p0, p1)
