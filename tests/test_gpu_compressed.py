"""Compressed particle storage on the GPU (Sec. 3.4, memory): positions as 32-bit fixed-point
coordinates and velocities as FP32, through the C ABI, against the oracle.

Expected results:
* fmm_compute_forces_i32 is bit for bit fmm_compute_forces on the FP64 positions u * 2^-32 (the
  conversion is exact, and everything after it is the same path), eager and replayed, isolated and
  periodic;
* fmm_kick_drift_i32 is the oracle's compressed substep exactly: integer positions, FP32
  velocities, rungs and active flags (both sides round each FP64 product and sum once, and round
  the drift to the nearest integer, ties to even); in the periodic box positions wrap, in the
  isolated box a particle that would leave stays and the next solve reports FMM_ERR_ARG;
* the context reports the device memory it holds.
"""
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


def ti32(u):
    """uint32 coordinates as the int32 tensor the binding passes on (same bits)."""
    return t(np.ascontiguousarray(u, dtype=np.uint32).view(np.int32), torch.int32)


def u32(tensor):
    return tensor.cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("nrep", [0, 1])
def test_fixed_point_solve_is_the_fp64_solve(ctx, nrep):
    n = 30000
    pos, mass = synth.clustered_nfw(n, 31)
    u = kdk.to_fixed(pos)
    x = kdk.from_fixed(u)
    eps, theta = synth.paper_softening(n), 0.55
    ctx.set_params(nrep=nrep)
    outs = []
    tu, tx, tm = ti32(u), t(x, torch.float64), t(mass, torch.float32)
    a = torch.zeros(3 * n, dtype=torch.float32, device="cuda:0")
    p = torch.zeros(n, dtype=torch.float32, device="cuda:0")
    try:
        for graphs in (False, True):
            ctx.set_graphs(graphs)
            for i32 in (False, True):
                for _ in range(2 if graphs else 1):  # with graphs: capture, then replay
                    a.fill_(float("nan"))
                    p.fill_(float("nan"))
                    if i32:
                        ctx.compute_forces_i32(tu, tm, eps, theta, a, p)
                    else:
                        ctx.compute_forces(tx, tm, eps, theta, a, p)
                    torch.cuda.synchronize()
                    outs.append((a.cpu().numpy(), p.cpu().numpy()))
        assert ctx.graph_info()["replays"] >= 1
    finally:
        ctx.set_graphs(False)
        ctx.set_params(nrep=0)
    for a, p in outs[1:]:
        assert np.array_equal(a, outs[0][0]) and np.array_equal(p, outs[0][1])
    # and the solve is accurate: against the FP64 direct sum at 512 sinks (isolated box)
    if nrep == 0:
        sinks = np.arange(0, n, n // 512)
        ref, _ = oracle.direct(x, mass, eps, sinks)
        a = outs[0][0].reshape(3, n)[:, sinks].astype(np.float64)
        e = np.linalg.norm(a - ref, axis=0) / np.linalg.norm(ref, axis=0)
        assert float(np.sqrt(np.mean(e * e))) <= 1e-3


@pytest.mark.parametrize("periodic", [False, True])
def test_fixed_point_kick_drift_is_the_oracle_substep(ctx, periodic):
    rng = np.random.default_rng(41)
    n = 40000
    u = rng.integers(0, 2 ** 32, (3, n), dtype=np.uint64).astype(np.uint32)
    if not periodic:  # away from the walls: none leaves in 8 substeps
        u = kdk.to_fixed(0.1 + 0.8 * kdk.from_fixed(u))
    vel = (0.5 * rng.standard_normal((3, n))).astype(np.float32)
    acc = (rng.standard_normal((3, n)) * 10.0 ** rng.uniform(-1, 3, n)).astype(np.float32)
    R, eps, dt0 = 3, 1e-3, 2e-3
    rung = rng.integers(0, R + 1, n)
    ctx.set_params(nrep=1 if periodic else 0)
    tu, tv = ti32(u), t(vel, torch.float32)
    tr = t(rung.astype(np.uint8), torch.uint8)
    act = torch.zeros(n, dtype=torch.uint8, device="cuda:0")
    ta = t(acc, torch.float32)
    try:
        for s in range(8):
            closing = s > 0
            u, vel, rung, an, out = kdk.kick_drift_i32(u, vel, acc, rung, eps, dt0, R, s, closing, periodic=periodic)
            ctx.kick_drift_i32(tu, tv, ta, tr, act, eps, dt0, R, s, closing)
            torch.cuda.synchronize()
            assert not out.any()
            assert np.array_equal(u32(tu).reshape(3, n), u), s
            assert np.array_equal(tv.cpu().numpy().reshape(3, n), vel), s
            assert np.array_equal(tr.cpu().numpy().astype(np.int64), rung), s
            assert np.array_equal(act.cpu().numpy().astype(bool), an), s
    finally:
        ctx.set_params(nrep=0)
    if periodic:
        # the wrap moved particles across the faces, which the fixed-point solve takes as it is
        a = torch.zeros(3 * n, dtype=torch.float32, device="cuda:0")
        ctx.set_params(nrep=1)
        try:
            ctx.compute_forces_i32(tu, t(np.full(n, 1.0 / n, np.float32), torch.float32), eps, 0.55, a)
            torch.cuda.synchronize()
        finally:
            ctx.set_params(nrep=0)
        assert np.all(np.isfinite(a.cpu().numpy()))


def test_isolated_box_keeps_a_leaving_particle_and_reports_it(ctx):
    n = 1000
    pos, mass = synth.clustered_plummer(n, 51)
    u = kdk.to_fixed(pos)
    u[0, 5] = 2 ** 32 - 3  # at the upper x face, moving out
    vel = np.zeros((3, n), np.float32)
    vel[0, 5] = 1.0
    h = 1e-3
    tu, tv = ti32(u), t(vel, torch.float32)
    acc = torch.zeros(3 * n, dtype=torch.float32, device="cuda:0")
    rung = torch.zeros(n, dtype=torch.uint8, device="cuda:0")
    act = torch.zeros(n, dtype=torch.uint8, device="cuda:0")
    ctx.kick_drift_i32(tu, tv, acc, rung, act, 1e-3, h, 0, 0, False)
    torch.cuda.synchronize()
    got = u32(tu).reshape(3, n)
    assert got[0, 5] == 2 ** 32 - 3 and np.all(got[:, 5] == u[:, 5])
    want, _, _, _, out = kdk.kick_drift_i32(u, vel, np.zeros((3, n), np.float32), np.zeros(n, int), 1e-3, h, 0, 0,
                                            False)
    assert out[5] and np.array_equal(got, want)
    with pytest.raises(binding.FmmError) as ei:
        ctx.compute_forces_i32(tu, t(mass, torch.float32), 1e-3, 0.7, acc)
    assert ei.value.status == -1
    # reported once: the context solves again
    ctx.compute_forces_i32(tu, t(mass, torch.float32), 1e-3, 0.7, acc)
    torch.cuda.synchronize()
    assert np.all(np.isfinite(acc.cpu().numpy()))


def test_memory_info_counts_the_buffers(ctx):
    fresh = binding.Context(0)
    try:
        d0, _ = fresh.memory_info()
        n = 200000
        pos, mass = synth.clustered_plummer(n, 61)
        free0, _ = torch.cuda.mem_get_info()
        acc = torch.zeros(3 * n, dtype=torch.float32, device="cuda:0")
        fresh.compute_forces_i32(ti32(kdk.to_fixed(pos)), t(mass, torch.float32), 1e-3, 0.7, acc)
        torch.cuda.synchronize()
        d1, h1 = fresh.memory_info()
        free1, _ = torch.cuda.mem_get_info()
        assert d1 > d0 and h1 > 0
        # what the context reports is what the device lost, within the torch tensors of this test
        # and the allocator's rounding (2 MB pages)
        lost = free0 - free1 - 3 * n * 4 - 3 * n * 4 - n * 4
        assert abs(lost - d1) <= 0.1 * d1 + (64 << 20), (lost, d1)
        print(f"\ncontext device bytes per particle at n = {n}: {d1 / n:.0f}")
    finally:
        fresh.close()
