"""Pins of the oracle's rung / kick-drift-kick schedule (Sec. 3.2) against closed forms:
a softened two-body circular orbit, time reversibility, the single-rung special case (the
textbook leapfrog) and the rung thresholds and synchronisation rule."""
import math

import numpy as np
import pytest

import oracle
from oracle import kdk


def _direct_force(mass, eps):
    def f(pos, act):
        acc, _ = oracle.direct(pos, mass, eps)
        return acc.astype(np.float32)
    return f


def _two_body(d=0.1, m=0.5, eps=0.005):
    v = math.sqrt(m * d * d / (2.0 * (d * d + eps * eps) ** 1.5))  # circular: v^2/(d/2) = m d/(d^2+eps^2)^1.5
    pos = np.array([[0.5 - d / 2, 0.5 + d / 2], [0.5, 0.5], [0.5, 0.5]])
    vel = np.array([[0.0, 0.0], [-v, v], [0.0, 0.0]])
    period = 2 * math.pi * (d / 2) / v
    return pos, vel, np.array([m, m]), eps, period


def _energy(pos, vel, mass, eps):
    _, phi = oracle.direct(pos, mass, eps)
    return 0.5 * float((mass * (vel ** 2).sum(axis=0)).sum()) + 0.5 * float((mass * phi).sum())


def test_two_body_circular_orbit_period_and_energy():
    pos, vel, mass, eps, period = _two_body()
    steps = 256
    dt0 = period / steps
    e0 = _energy(pos, vel, mass, eps)
    p, v, r, acc = kdk.run(pos, vel, mass, eps, dt0, 0, steps, _direct_force(mass, eps), rung=np.zeros(2, int))
    v = kdk.close(v, acc, r, dt0)
    # back where it started after one period (leapfrog phase error is O(dt^2))
    assert np.abs(p - pos).max() < 1e-3 * 0.1
    assert abs(_energy(p, v, mass, eps) / e0 - 1) < 1e-4


def test_single_rung_is_the_textbook_leapfrog():
    pos, vel, mass, eps, period = _two_body()
    dt = period / 40
    f = _direct_force(mass, eps)
    p, v, r, acc = kdk.run(pos, vel, mass, eps, dt, 0, 7, f, rung=np.zeros(2, int))
    v = kdk.close(v, acc, r, dt)
    # kick-drift-kick: v(n+1/2) = v(n) + a(n) dt/2, x(n+1) = x(n) + v(n+1/2) dt, v(n+1) = v(n+1/2) + a(n+1) dt/2
    x, u = pos.copy(), vel.copy()
    a = f(x, None).astype(np.float64)
    for _ in range(7):
        u = u + a * dt / 2
        x = x + u * dt
        a = f(x, None).astype(np.float64)
        u = u + a * dt / 2
    assert np.allclose(p, x, rtol=0, atol=1e-15) and np.allclose(v, u, rtol=0, atol=1e-13)


def test_time_reversibility_on_one_rung():
    pos, vel, mass, eps, period = _two_body()
    dt = period / 50
    f = _direct_force(mass, eps)
    p, v, r, acc = kdk.run(pos, vel, mass, eps, dt, 0, 20, f, rung=np.zeros(2, int))
    v = kdk.close(v, acc, r, dt)
    p2, v2, r2, acc2 = kdk.run(p, -v, mass, eps, dt, 0, 20, f, rung=np.zeros(2, int))
    v2 = kdk.close(v2, acc2, r2, dt)
    assert np.abs(p2 - pos).max() < 1e-12 and np.abs(v2 + vel).max() < 1e-10


def test_rung_thresholds_and_synchronisation():
    eps, dt0, R = 1e-3, 1.0, 4
    # |a| such that Delta T = 0.2 sqrt(eps/|a|) equals dt0 / 2^k exactly -> rung k; slightly below -> k + 1
    ks = np.arange(0, 4)
    amag = eps * (0.2 * np.ldexp(1.0, ks)) ** 2 / dt0 ** 2
    acc = np.zeros((3, 2 * len(ks)), np.float32)
    acc[0, : len(ks)] = amag.astype(np.float32)
    acc[0, len(ks):] = (amag * 1.001).astype(np.float32)
    r = kdk.target_rungs(acc, eps, dt0, R)
    dts = kdk.timestep(acc, eps)
    for i in range(acc.shape[1]):
        rr = int(r[i])
        assert dt0 / 2 ** rr <= dts[i] and (rr == 0 or dt0 / 2 ** (rr - 1) > dts[i])
    assert kdk.target_rungs(np.zeros((3, 1), np.float32), eps, dt0, R)[0] == 0
    # a particle on rung 3 at substep 2 (R = 3) that wants rung 0 may only reach rung 2
    pos = np.full((3, 1), 0.5)
    vel = np.zeros((3, 1))
    _, _, rung, act = kdk.kick_drift(pos, vel, np.zeros((3, 1), np.float32), np.array([3]), eps, 1.0, 3, 2, True)
    assert rung[0] == 2 and act[0] == False  # rung 2 is next active at substep 4
    _, _, rung, act = kdk.kick_drift(pos, vel, np.zeros((3, 1), np.float32), np.array([3]), eps, 1.0, 3, 4, True)
    assert rung[0] == 1


# ---------------------------------------------------------------- compressed storage (Sec. 3.4)


def test_compressed_substep_is_the_fp64_substep_rounded():
    """One substep on 32-bit positions and FP32 velocities lands within the rounding of that storage
    of the FP64 substep: |dx| <= |v64 - v32| h + 2^-33 (the drift's rounding to the grid) + 2^-52 (the
    FP64 substep's own rounding of x + v h, x < 1), and the velocity is the FP64 one rounded to FP32."""
    rng = np.random.default_rng(3)
    n = 500
    pos = kdk.from_fixed(kdk.to_fixed(0.2 + 0.6 * rng.random((3, n))))
    vel32 = (0.3 * rng.standard_normal((3, n))).astype(np.float32)
    acc = (5.0 * rng.standard_normal((3, n))).astype(np.float32)
    rung = rng.integers(0, 4, n)
    eps, dt0, R = 1e-3, 1e-3, 3
    for s in range(8):
        p64, v64, r64, a64 = kdk.kick_drift(pos, vel32.astype(np.float64), acc, rung, eps, dt0, R, s, s > 0)
        u, v, r, a, out = kdk.kick_drift_i32(kdk.to_fixed(pos), vel32, acc, rung, eps, dt0, R, s, s > 0)
        assert not out.any() and np.array_equal(r, r64) and np.array_equal(a, a64)
        assert np.array_equal(v, v64.astype(np.float32))
        h = math.ldexp(dt0, -R)
        bound = np.abs(v64 - v.astype(np.float64)) * h + 2.0 ** -33 + 2.0 ** -52
        assert np.all(np.abs(kdk.from_fixed(u) - p64) <= bound)


def test_compressed_drift_wraps_in_the_periodic_box_and_stops_at_the_isolated_walls():
    # u = 2^32 - 10 moving by +25 units of 2^-32 per substep: 15 in the periodic box
    h = 2.0 ** -30  # dt0 with R = 0
    ipos = np.array([[2 ** 32 - 10], [7], [2 ** 31]], dtype=np.uint32)
    vel = np.array([[25.0 * 2.0 ** -32 / h], [-8.0 * 2.0 ** -32 / h], [0.0]], dtype=np.float32)
    acc = np.zeros((3, 1), np.float32)
    u, v, r, a, out = kdk.kick_drift_i32(ipos, vel, acc, np.zeros(1, int), 1e-3, h, 0, 0, False, periodic=True)
    assert list(u[:, 0]) == [15, 2 ** 32 - 1, 2 ** 31] and not out[0]
    u, v, r, a, out = kdk.kick_drift_i32(ipos, vel, acc, np.zeros(1, int), 1e-3, h, 0, 0, False, periodic=False)
    assert out[0] and np.array_equal(u, ipos)


def test_compressed_storage_keeps_the_two_body_orbit():
    """The paper checked that the compression does not affect trajectories significantly: over one
    period of the softened circular orbit, 32-bit positions and FP32 velocities stay within 1e-6 of
    the box of the FP64 integration, and the energy error stays the leapfrog's."""
    pos, vel, mass, eps, period = _two_body()
    steps = 256
    dt0 = period / steps
    f = _direct_force(mass, eps)
    p64, v64, r, acc = kdk.run(pos, vel, mass, eps, dt0, 0, steps, f, rung=np.zeros(2, int))
    u = kdk.to_fixed(pos)
    v = vel.astype(np.float32)
    rung = np.zeros(2, int)
    a = f(kdk.from_fixed(u), None)
    for k in range(steps):
        u, v, rung, act, out = kdk.kick_drift_i32(u, v, a, rung, eps, dt0, 0, 0, k > 0)
        assert not out.any()
        a = f(kdk.from_fixed(u), None)
    assert np.abs(kdk.from_fixed(u) - p64).max() < 1e-6
    e0 = _energy(pos, vel, mass, eps)
    vc = kdk.close(v.astype(np.float64), a, rung, dt0)
    assert abs(_energy(kdk.from_fixed(u), vc, mass, eps) / e0 - 1) < 1e-4
