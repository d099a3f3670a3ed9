"""Parity of fmm_kick_drift / fmm_assign_rungs with the oracle's KDK schedule (Sec. 3.2).

Rungs and active flags are integers decided in FP64 with the same operation order on both
sides: exact.  Positions and velocities are FP64 updates v += a dt, x += v h that may differ by
the rounding of one fused multiply-add: relative 1e-15."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from oracle import kdk
from paper_1609_08621_gb300 import binding, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = binding.Context(0)
    yield c
    c.close()


def t(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a).reshape(-1)).to("cuda:0", dtype)


def test_assign_rungs_exact(ctx):
    rng = np.random.default_rng(4)
    n = 100000
    acc = (rng.standard_normal((3, n)) * 10.0 ** rng.uniform(-2, 4, n)).astype(np.float32)
    acc[:, :10] = 0.0
    eps, dt0, R = 1.5e-4, 0.05, 5
    r = torch.zeros(n, dtype=torch.uint8, device="cuda:0")
    ctx.assign_rungs(t(acc, torch.float32), r, eps, dt0, R)
    assert np.array_equal(r.cpu().numpy().astype(np.int64), kdk.target_rungs(acc, eps, dt0, R))


@pytest.mark.parametrize("s,closing", [(0, 0), (1, 1), (2, 1), (4, 1), (7, 1)])
def test_kick_drift_step_matches_oracle(ctx, s, closing):
    rng = np.random.default_rng(10 + s)
    n = 50000
    pos = 0.25 + 0.5 * rng.random((3, n))
    vel = 1e-3 * rng.standard_normal((3, n))
    acc = (rng.standard_normal((3, n)) * 10.0 ** rng.uniform(-1, 3, n)).astype(np.float32)
    R = 3
    rung = rng.integers(0, R + 1, n)
    eps, dt0 = 1e-3, 1e-3
    tp, tv, tr = t(pos, torch.float64), t(vel, torch.float64), t(rung, torch.uint8)
    an = torch.zeros(n, dtype=torch.uint8, device="cuda:0")
    ctx.kick_drift(tp, tv, t(acc, torch.float32), tr, an, eps, dt0, R, s, closing)
    torch.cuda.synchronize()
    p2, v2, r2, a2 = kdk.kick_drift(pos, vel, acc, rung, eps, dt0, R, s, closing)
    assert np.array_equal(tr.cpu().numpy().astype(np.int64), r2)
    assert np.array_equal(an.cpu().numpy().astype(bool), a2)
    assert np.allclose(tv.cpu().numpy().reshape(3, n), v2, rtol=1e-15, atol=1e-18)
    assert np.allclose(tp.cpu().numpy().reshape(3, n), p2, rtol=1e-15, atol=1e-18)


def test_hierarchical_run_with_fmm_forces_tracks_oracle(ctx):
    """8 substeps of the rung hierarchy on a clustered set: GPU forces + GPU kick-drift against the
    oracle's direct-sum forces + oracle schedule.  Rungs are decided from forces that differ by the
    method's truncation error, so a few particles may take a neighbouring rung; trajectories agree
    to the size of the force error times dt^2."""
    n, R = 3000, 3
    pos, mass = synth.clustered_plummer(n, 21)
    eps, theta = 1e-3, 0.55
    tp, tm = t(pos, torch.float64), t(mass, torch.float32)
    vel = torch.zeros(3 * n, dtype=torch.float64, device="cuda:0")
    acc = torch.zeros(3 * n, dtype=torch.float32, device="cuda:0")
    rung = torch.zeros(n, dtype=torch.uint8, device="cuda:0")
    act = torch.ones(n, dtype=torch.uint8, device="cuda:0")
    ctx.compute_forces(tp, tm, eps, theta, acc)
    a0 = acc.cpu().numpy().reshape(3, n)
    dt0 = float(np.ldexp(np.quantile(kdk.timestep(a0, eps), 0.1), R))
    ctx.assign_rungs(acc, rung, eps, dt0, R)
    for k in range(2 ** R):
        ctx.kick_drift(tp, vel, acc, rung, act, eps, dt0, R, k, 1 if k > 0 else 0)
        ctx.compute_forces(tp, tm, eps, theta, acc, None, act)
    torch.cuda.synchronize()
    gp = tp.cpu().numpy().reshape(3, n)

    def force(p, a):
        return oracle.direct(p, mass, eps)[0].astype(np.float32)

    op, ov, orung, oacc = kdk.run(pos, np.zeros((3, n)), mass, eps, dt0, R, 2 ** R, force)
    disp = np.abs(op - pos).max()
    assert disp > 0
    assert np.abs(gp - op).max() <= 2e-2 * disp
    assert np.mean(rung.cpu().numpy().astype(np.int64) == orung) > 0.99
