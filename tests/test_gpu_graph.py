"""The CUDA-graph solve: replays give results bit-identical to eager solves, follow changing
buffer contents, recapture when an argument changes, and fall back to an eager solve when the
captured levels or capacities are not enough."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1609_08621_gb300 import binding, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def t(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a).reshape(-1)).to("cuda:0", dtype)


def eager(pos, mass, eps, theta, **params):
    c = binding.Context(0, **params)
    try:
        n = mass.size
        acc = torch.zeros(3 * n, dtype=torch.float32, device="cuda:0")
        pot = torch.zeros(n, dtype=torch.float32, device="cuda:0")
        c.compute_forces(t(pos, torch.float64), t(mass, torch.float32), eps, theta, acc, pot)
        return acc.cpu().numpy(), pot.cpu().numpy(), c.stats()
    finally:
        c.close()


def test_replay_matches_eager_and_follows_buffer_contents(dev):
    n, eps, theta = 30000, 1e-3, 0.6
    p1, m1 = synth.clustered_plummer(n, 41)
    p2, m2 = synth.clustered_plummer(n, 42)
    c = binding.Context(0)
    try:
        c.set_graphs(True)
        tp, tm = t(p1, torch.float64), t(m1, torch.float32)
        acc = torch.zeros(3 * n, dtype=torch.float32, device=dev)
        pot = torch.zeros(n, dtype=torch.float32, device=dev)
        c.compute_forces(tp, tm, eps, theta, acc, pot)  # eager, captures
        assert c.graph_info()["captured"]
        for _ in range(2):
            acc.zero_()
            c.compute_forces(tp, tm, eps, theta, acc, pot)  # replays
        info = c.graph_info()
        assert info["replays"] == 2
        ea, ep, est = eager(p1, m1, eps, theta)
        assert np.array_equal(acc.cpu().numpy(), ea) and np.array_equal(pot.cpu().numpy(), ep)
        st = c.stats()
        for k in ("n_cells", "n_groups", "n_pp_pairs", "n_pc_pairs", "n_cc", "n_cp", "n_levels"):
            assert st[k] == est[k], k
        assert st["n_launches"] > 50 and st["ms_total"] > 0
        # new contents in the same buffers: still a replay, still the eager result
        tp.copy_(t(p2, torch.float64))
        tm.copy_(t(m2, torch.float32))
        c.compute_forces(tp, tm, eps, theta, acc, pot)
        assert c.graph_info()["replays"] == 3
        ea2, ep2, _ = eager(p2, m2, eps, theta)
        assert np.array_equal(acc.cpu().numpy(), ea2) and np.array_equal(pot.cpu().numpy(), ep2)
        # another theta: eager solve and a new capture
        c.compute_forces(tp, tm, eps, 0.5, acc, pot)
        assert c.graph_info()["replays"] == 3 and c.graph_info()["captured"]
        ea3, _, _ = eager(p2, m2, eps, 0.5)
        assert np.array_equal(acc.cpu().numpy(), ea3)
        c.set_graphs(False)
        assert not c.graph_info()["captured"]
    finally:
        c.close()


def test_replay_falls_back_when_the_tree_is_deeper(dev):
    """Capture on a uniform box, then put a tightly clustered set into the same buffers: its tree
    is far deeper than the captured levels, so the replay must hand over to an eager solve."""
    n, eps, theta = 20000, 1e-4, 0.6
    pu, mu = synth.uniform_box(n, 51)
    pc, mc = synth.clustered_plummer(n, 52, n_spheres=1, scale=1e-4, uniform_frac=0.0)
    c = binding.Context(0)
    try:
        c.set_graphs(True)
        tp, tm = t(pu, torch.float64), t(mu, torch.float32)
        acc = torch.zeros(3 * n, dtype=torch.float32, device=dev)
        c.compute_forces(tp, tm, eps, theta, acc)
        levels_uniform = c.stats()["n_levels"]
        tp.copy_(t(pc, torch.float64))
        tm.copy_(t(mc, torch.float32))
        c.compute_forces(tp, tm, eps, theta, acc)
        assert c.stats()["n_levels"] > levels_uniform + 5
        ea, _, _ = eager(pc, mc, eps, theta)
        assert np.array_equal(acc.cpu().numpy(), ea)
        # the eager repeat captured a graph for the deeper tree; it now replays
        before = c.graph_info()["replays"]
        c.compute_forces(tp, tm, eps, theta, acc)
        assert c.graph_info()["replays"] == before + 1
        assert np.array_equal(acc.cpu().numpy(), ea)
    finally:
        c.close()


def test_batch_solves_replay(dev):
    boxes, off = synth.batch_boxes(6, 61)
    pos = np.concatenate([b[0] for b in boxes], axis=1)
    mass = np.concatenate([b[1] for b in boxes])
    n = mass.size
    c = binding.Context(0)
    try:
        c.set_graphs(True)
        tp, tm = t(pos, torch.float64), t(mass, torch.float32)
        acc = torch.zeros(3 * n, dtype=torch.float32, device=dev)
        pot = torch.zeros(n, dtype=torch.float32, device=dev)
        c.compute_forces_batch(tp, tm, off, 1e-3, 0.7, acc, pot)
        first = acc.cpu().numpy()
        c.compute_forces_batch(tp, tm, off, 1e-3, 0.7, acc, pot)
        assert c.graph_info()["replays"] == 1
        assert np.array_equal(acc.cpu().numpy(), first)
    finally:
        c.close()


def test_learned_criterion_replays(dev):
    """A graph captured with the learned criterion (its walk mode and the per-cell acceleration
    scale) replays to the eager result."""
    from oracle import mlp as omlp

    n, eps, theta = 20000, 1e-3, 0.55
    pos, mass = synth.clustered_plummer(n, 71)
    rng = np.random.default_rng(5)
    flat = np.zeros(omlp.N_PARAMS)
    flat[:omlp.N_WEIGHTS] = 0.1 * rng.standard_normal(omlp.N_WEIGHTS)
    p = omlp.unpack(flat)
    p["b4"][:] = -4.0
    p["inv_std"][:] = 1.0
    params = omlp.pack(p).astype(np.float32)
    tp, tm = t(pos, torch.float64), t(mass, torch.float32)
    est = torch.zeros(3 * n, dtype=torch.float32, device=dev)
    c0 = binding.Context(0)
    try:  # the acceleration estimate: a fixed-theta solve
        c0.compute_forces(tp, tm, eps, theta, est)
    finally:
        c0.close()
    outs = []
    for graphs in (False, True):
        c = binding.Context(0)
        try:
            c.mlp_load(params)
            c.set_params(criterion=1, mlp_tau=-3.5)
            c.set_graphs(graphs)
            acc = torch.zeros(3 * n, dtype=torch.float32, device=dev)
            for _ in range(3):
                acc.copy_(est)
                c.compute_forces(tp, tm, eps, theta, acc)
            if graphs:
                assert c.graph_info()["replays"] == 2
            assert c.stats()["n_learned"] > 0
            outs.append(acc.cpu().numpy())
        finally:
            c.close()
    assert np.array_equal(outs[0], outs[1])


def test_autotune_over_a_batch(dev):
    boxes, off = synth.batch_boxes(5, 72)
    pos = np.concatenate([b[0] for b in boxes], axis=1)
    mass = np.concatenate([b[1] for b in boxes])
    n = mass.size
    c = binding.Context(0)
    try:
        acc = torch.zeros(3 * n, dtype=torch.float32, device=dev)
        best, ms = c.autotune(t(pos, torch.float64), t(mass, torch.float32), 1e-3, 0.7, acc,
                              candidates=[(16, 64, 64), (8, 32, 128)], reps=1, box_offsets=off)
        assert (best.bucket, best.group, best.list_chunk) in [(16, 64, 64), (8, 32, 128)] and ms > 0
    finally:
        c.close()
