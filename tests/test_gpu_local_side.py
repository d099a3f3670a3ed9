"""The local expansions of each walk level on a side stream, beside the levels below (the path
large walks take), against the same expansions after the last level (the path small walks take).

Every sink's M2L and P2L terms are added in its own list order by one warp in both, and the top-down
pass runs level by level in both, so the forces must agree bit for bit: eager solves, CUDA-graph
replays, the periodic box and the learned criterion's walk.  fmm_debug_local_side(0) makes every
walk after a context's first take the side stream.
"""
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


def solves(ctx, pos, mass, eps, theta, k):
    """k solves into the same output buffers (a graph replays only at the addresses it captured)."""
    n = mass.size
    tp, tm = t(pos, torch.float64), t(mass, torch.float32)
    acc = torch.zeros(3 * n, dtype=torch.float32, device="cuda:0")
    pot = torch.zeros(n, dtype=torch.float32, device="cuda:0")
    out = []
    for _ in range(k):
        acc.zero_()
        pot.zero_()
        ctx.compute_forces(tp, tm, eps, theta, acc, pot)
        torch.cuda.synchronize()
        out.append((acc.cpu().numpy(), pot.cpu().numpy()))
    return out


@pytest.mark.parametrize("graphs,nrep", [(False, 0), (True, 0), (False, 1)])
def test_side_stream_gives_the_bits_of_the_in_order_path(dev, graphs, nrep):
    n = 262144
    pos, mass = synth.make("nfw", n, 5)
    eps, theta = synth.paper_softening(n), 0.55
    params = dict(bucket=16, group=64, list_chunk=128)
    if nrep:
        params["nrep"] = nrep
    ref = binding.Context(0, **params)
    side = binding.Context(0, **params)
    try:
        ref.set_graphs(graphs)
        side.set_graphs(graphs)
        side.debug_local_side(0)
        r = solves(ref, pos, mass, eps, theta, 4)
        s = solves(side, pos, mass, eps, theta, 4)
        assert side.stats()["n_cc"] > 0
        if not graphs:
            # the side stream launches M2L, P2L and L2L per level: more kernels than the in-order path
            assert side.stats()["n_launches"] > ref.stats()["n_launches"]
        for (ra, rp), (sa, sp) in zip(r, s):
            assert np.array_equal(ra, sa) and np.array_equal(rp, sp)
        if graphs:
            assert side.graph_info()["replays"] >= 1  # the later solves replayed a captured graph
    finally:
        ref.close()
        side.close()


def _random_params(seed):
    from oracle import mlp as omlp

    rng = np.random.default_rng(seed)
    flat = np.zeros(omlp.N_PARAMS)
    flat[:omlp.N_WEIGHTS] = 0.25 * rng.standard_normal(omlp.N_WEIGHTS)
    p = omlp.unpack(flat)
    p["mean"][:] = rng.standard_normal(8)
    p["inv_std"][:] = 0.5 + rng.random(8)
    return omlp.pack(p).astype(np.float32)


def test_side_stream_learned_walk(dev):
    """The learned criterion's walk (untrained weights: only the two orders are compared), with
    the acceleration estimate of a fixed-theta solve."""
    n = 65536
    pos, mass = synth.make("nfw", n, 9)
    eps, theta = synth.paper_softening(n), 0.55
    tp, tm = t(pos, torch.float64), t(mass, torch.float32)
    ref = binding.Context(0, bucket=16, group=64)
    side = binding.Context(0, bucket=16, group=64)
    try:
        est = torch.zeros(3 * n, dtype=torch.float32, device="cuda:0")
        ref.compute_forces(tp, tm, eps, theta, est)
        w = _random_params(3)
        outs = {}
        for name, c in (("ref", ref), ("side", side)):
            c.mlp_load(w)
            if name == "side":
                c.debug_local_side(0)
            c.set_params(criterion=1, mlp_tau=-3.5)
            res = []
            for _ in range(3):
                acc = est.clone()
                c.compute_forces(tp, tm, eps, theta, acc)
                torch.cuda.synchronize()
                res.append(acc.cpu().numpy())
            outs[name] = res
            assert c.stats()["n_learned"] > 0
        assert side.stats()["n_launches"] > ref.stats()["n_launches"]
        for ra, sa in zip(outs["ref"], outs["side"]):
            assert np.array_equal(ra, sa)
    finally:
        ref.close()
        side.close()
