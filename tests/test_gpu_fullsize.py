"""The measured workloads at full size, in the launch configuration that bench.py times.

That configuration is buckets of 16, groups of 64 and work items of 128 list entries, and every
solve after the first is a CUDA-graph replay. Each test:
- checks that the replay is bit-identical to the eager solve that captured it;
- checks sampled sinks against the oracle's FP64 direct sum, to the method's accuracy target
  (rms relative force error <= 1e-3, 99th percentile <= 1e-2).

The sinks are few enough that the direct sum takes seconds on the host cores.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1609_08621_gb300 import binding, synth

pytestmark = pytest.mark.gpu

BENCH_PARAMS = dict(bucket=16, group=64, list_chunk=128)


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = binding.Context(0, **BENCH_PARAMS)
    c.set_graphs(True)
    yield c
    c.close()


def _t(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a).reshape(-1)).to("cuda:0", dtype)


def _rel_err(a, ref):
    return np.linalg.norm(a - ref, axis=0) / np.linalg.norm(ref, axis=0)


def _assert_accuracy(e):
    rms = float(np.sqrt(np.mean(np.square(e))))
    p99 = float(np.quantile(e, 0.99))
    assert rms <= 1e-3 and p99 <= 1e-2, (rms, p99)


def _eager_then_replay(ctx, solve, acc, pot):
    """Run solve() twice on the same buffers: the first call solves eagerly and captures a graph,
    the second replays it. Return the replayed result after checking it equals the eager one."""
    acc.fill_(float("nan"))
    pot.fill_(float("nan"))
    solve()
    a0, p0 = acc.cpu().numpy().copy(), pot.cpu().numpy().copy()
    replays = ctx.graph_info()["replays"]
    acc.fill_(float("nan"))
    pot.fill_(float("nan"))
    solve()
    assert ctx.graph_info()["replays"] == replays + 1
    a1, p1 = acc.cpu().numpy(), pot.cpu().numpy()
    assert np.array_equal(a0, a1, equal_nan=True) and np.array_equal(p0, p1, equal_nan=True)
    return a1, p1


def test_nfw_128cubed(ctx):
    n = 128 ** 3
    pos, mass = synth.clustered_nfw(n, 2)
    eps, theta = synth.paper_softening(n), 0.55
    tp, tm = _t(pos, torch.float64), _t(mass, torch.float32)
    acc = torch.empty(3 * n, dtype=torch.float32, device="cuda:0")
    pot = torch.empty(n, dtype=torch.float32, device="cuda:0")
    a, p = _eager_then_replay(ctx, lambda: ctx.compute_forces(tp, tm, eps, theta, acc, pot), acc, pot)
    a = a.reshape(3, n).astype(np.float64)
    assert np.all(np.isfinite(a)) and np.all(np.isfinite(p))
    sinks = np.random.default_rng(11).choice(n, 2048, replace=False)
    ref, rp = oracle.direct(pos, mass, eps, sinks)
    _assert_accuracy(_rel_err(a[:, sinks], ref))
    ep = np.abs(p[sinks] - rp) / np.abs(rp)
    assert float(np.sqrt(np.mean(ep ** 2))) <= 1e-3


def test_batch_of_64_boxes(ctx):
    boxes, off = synth.batch_boxes(64, 3)
    pos = np.concatenate([b[0] for b in boxes], axis=1)
    mass = np.concatenate([b[1] for b in boxes])
    n = mass.size
    eps, theta = 1e-3, 0.7
    tp, tm = _t(pos, torch.float64), _t(mass, torch.float32)
    acc = torch.empty(3 * n, dtype=torch.float32, device="cuda:0")
    pot = torch.empty(n, dtype=torch.float32, device="cuda:0")
    a, p = _eager_then_replay(ctx, lambda: ctx.compute_forces_batch(tp, tm, off, eps, theta, acc, pot), acc, pot)
    a = a.reshape(3, n).astype(np.float64)
    assert np.all(np.isfinite(a))
    rng = np.random.default_rng(12)
    errs = []
    for b, (pb, mb) in enumerate(boxes):
        local = rng.choice(mb.size, 32, replace=False)
        ref, _ = oracle.direct(pb, mb, eps, local)  # the box's own particles are its only sources
        errs.append(_rel_err(a[:, off[b] + local], ref))
    _assert_accuracy(np.concatenate(errs))


def test_rungs_256cubed_active_subset(ctx):
    """The particles of the finest rung (about 10%, the active set of an odd substep) get forces;
    every other particle's outputs are left untouched."""
    n = 256 ** 3
    R = 5
    pos, mass = synth.clustered_plummer(n, 4)
    eps, theta = synth.paper_softening(n), 0.55
    tp, tm = _t(pos, torch.float64), _t(mass, torch.float32)
    acc = torch.empty(3 * n, dtype=torch.float32, device="cuda:0")
    pot = torch.empty(n, dtype=torch.float32, device="cuda:0")
    ctx.compute_forces(tp, tm, eps, theta, acc, pot)
    a_all = acc.cpu().numpy().reshape(3, n).astype(np.float64)
    dtp = 0.2 * np.sqrt(eps / np.maximum(np.linalg.norm(a_all, axis=0), 1e-30))
    dt0 = float(np.ldexp(np.quantile(dtp, 0.10), R - 1))
    rung = torch.zeros(n, dtype=torch.uint8, device="cuda:0")
    ctx.assign_rungs(acc, rung, eps, dt0, R)
    active = (rung == R).to(torch.uint8)
    frac = float(active.float().mean())
    assert 0.05 <= frac <= 0.2, frac
    a, p = _eager_then_replay(ctx, lambda: ctx.compute_forces(tp, tm, eps, theta, acc, pot, active), acc, pot)
    a = a.reshape(3, n)
    act = active.cpu().numpy().astype(bool)
    assert np.all(np.isnan(a[:, ~act])) and np.all(np.isnan(p[~act]))
    assert np.all(np.isfinite(a[:, act]))
    sinks = np.random.default_rng(13).choice(np.flatnonzero(act), 256, replace=False)
    ref, _ = oracle.direct(pos, mass, eps, sinks)
    _assert_accuracy(_rel_err(a[:, sinks].astype(np.float64), ref))


def test_nfw_128cubed_lists_and_locals_match_the_oracle(ctx):
    """The bench's 128^3 NFW box and settings with 4096 random active sinks on both sides (the tree
    is the whole box's, 37 levels deep): PP, PC, CC and CP list sets identical to the oracle's, and
    every group's local expansion (evaluated by the oracle's FP64 L2P at the group's active sinks)
    and PP + PC + local forces at FP32 tolerance of the oracle FMM's."""
    n = 128 ** 3
    pos, mass = synth.clustered_nfw(n, 2)
    eps, theta = synth.paper_softening(n), 0.55
    act = np.zeros(n, np.uint8)
    act[np.random.default_rng(17).choice(n, 4096, replace=False)] = 1
    tp, tm, ta = _t(pos, torch.float64), _t(mass, torch.float32), _t(act, torch.uint8)
    acc = torch.full((3 * n,), float("nan"), dtype=torch.float32, device="cuda:0")
    ctx.compute_forces(tp, tm, eps, theta, acc, None, ta)
    torch.cuda.synchronize()
    orc = oracle.FMM(pos, mass, eps, theta, bucket=16, group=64, active=act)
    g = ctx.export_cells()
    o = orc.cells()
    grng = np.stack([g["first"], g["count"]], axis=1)
    orng = np.stack([o["first"], o["count"]], axis=1)
    for kind in ("pp", "pc", "cc", "cp"):
        s, f, c = ctx.export_lists(kind)
        os_, of, oc = orc.entries(kind)
        gs = set(zip(map(tuple, grng[s]), f.tolist(), c.tolist()))
        ost = set(zip(map(tuple, orng[os_]), of.tolist(), oc.tolist()))
        assert len(gs) == len(s) and gs == ost, (kind, len(gs - ost), len(ost - gs))
    # group local expansions: matched by the group cell's particle range
    gcell, gL = ctx.export_locals()
    ocell, oL = orc.groups()
    # the GPU's coefficients in the oracle's multi-index order
    loc_idx, _ = binding.fmm_multi_index()
    mi = oracle.multi_index()
    gL = gL[:, [int(np.where((loc_idx == m).all(axis=1))[0][0]) for m in mi]]
    okey = {(int(o["first"][c]), int(o["count"][c])): i for i, c in enumerate(ocell)}
    perm = orc.perm()
    ra, _ = orc.forces()
    scale = np.linalg.norm(ra, axis=0)
    errs = []
    for i, c in enumerate(gcell):
        key = (int(g["first"][c]), int(g["count"][c]))
        j = okey[key]
        com = o["com"][ocell[j]]
        for q in range(key[0], key[0] + key[1]):
            p = int(perm[q])
            if not act[p]:
                continue
            u = pos[:, p] - com
            ag, _ = oracle.l2p(gL[i].astype(np.float64), u)
            ao, _ = oracle.l2p(oL[j], u)
            errs.append(np.linalg.norm(ag - ao) / scale[p])
    assert len(okey) == len(gcell) and len(errs) == int(act.sum())
    errs = np.array(errs)
    assert float(np.sqrt(np.mean(errs ** 2))) <= 2e-5 and errs.max() <= 2e-3
    a = acc.cpu().numpy().reshape(3, n).astype(np.float64)
    sel = act.astype(bool)
    e = np.linalg.norm(a[:, sel] - ra[:, sel], axis=0) / scale[sel]
    assert float(np.sqrt(np.mean(e ** 2))) <= 2e-5 and e.max() <= 2e-3
