"""Individual time steps on rungs with the hierarchical kick-drift-kick leapfrog -- FP64 oracle.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. 3.2: every particle's step is 2^-l of the base step dt0, l being its rung; a particle's
step is chosen from Delta T_i = 0.2 sqrt(eps / |a_i|); the leapfrog is kick-drift-kick in the
hierarchical arrangement of Fig. KDK, where the kicks of finer rungs line up with those of
coarser ones and only the particles whose kicks fall on a given substep (the active ones)
need new forces there.

Schedule (one base step = 2^R substeps of h = dt0 / 2^R; rung r is active at substep s when
s is a multiple of 2^(R - r)).  At substep s, for the active particles:
  1. closing half kick of the step that ends at s:  v += a dt0 / 2^(r+1)  (skipped at the very
     first substep of a run, where no step has started);
  2. new rung: the target rung is the smallest r in [0, R] with dt0 / 2^r <= Delta T
     (|a| = 0 gives rung 0); a particle may only move to a coarser rung r' at a substep where
     r' is synchronised (s a multiple of 2^(R - r')), otherwise it takes the coarsest
     synchronised rung that is not coarser than its target;
  3. opening half kick with the new rung:  v += a dt0 / 2^(r+1);
then every particle drifts, x += v h, and the particles active at s + 1 get new forces.
The rung choice is an integer decided by floating point; it is made in FP64 with the
operations in this order: a2 = (ax^2 + ay^2) + az^2 from the single-precision components,
|a| = sqrt(a2), Delta T = 0.2 * sqrt(eps / |a|), and the test dt0 > Delta T * 2^r.
"""
from __future__ import annotations

import math

import numpy as np


def timestep(acc, eps):
    """Delta T_i = 0.2 sqrt(eps / |a_i|) (Sec. 3.2); acc (3, N) single-precision components."""
    a = np.asarray(acc, dtype=np.float32).astype(np.float64)
    a2 = (a[0] * a[0] + a[1] * a[1]) + a[2] * a[2]
    am = np.sqrt(a2)
    with np.errstate(divide="ignore"):
        dt = 0.2 * np.sqrt(eps / am)
    dt[~(am > 0.0)] = np.inf
    return dt


def target_rungs(acc, eps, dt0, max_rung):
    """Smallest r in [0, max_rung] with dt0 / 2^r <= Delta T."""
    dt = timestep(acc, eps)
    r = np.zeros(dt.shape, dtype=np.int64)
    for k in range(max_rung):
        r += (dt0 > np.ldexp(dt, k)) & (r == k)
    return r


def active(rung, s, max_rung):
    period = np.left_shift(1, max_rung - np.asarray(rung, dtype=np.int64))
    return (s % period) == 0


def kick_drift(pos, vel, acc, rung, eps, dt0, max_rung, s, closing):
    """One substep; returns new (pos, vel, rung, active_next).  pos, vel (3, N) float64."""
    pos = np.array(pos, dtype=np.float64)
    vel = np.array(vel, dtype=np.float64)
    rung = np.array(rung, dtype=np.int64)
    a = np.asarray(acc, dtype=np.float32).astype(np.float64)
    act = active(rung, s, max_rung)
    if closing:
        vel[:, act] += a[:, act] * np.ldexp(dt0, -rung[act] - 1)
    tgt = target_rungs(acc, eps, dt0, max_rung)
    new = rung.copy()
    for i in np.nonzero(act)[0]:
        rt, r = int(tgt[i]), int(rung[i])
        if rt >= r:
            new[i] = rt
        else:
            rn = rt
            while rn < r and s % (1 << (max_rung - rn)) != 0:
                rn += 1
            new[i] = rn
    rung = new
    vel[:, act] += a[:, act] * np.ldexp(dt0, -rung[act] - 1)
    pos += vel * math.ldexp(dt0, -max_rung)
    return pos, vel, rung, active(rung, s + 1, max_rung)


def run(pos, vel, mass, eps, dt0, max_rung, n_substeps, force, rung=None):
    """Integrate n_substeps substeps from the start of a base step.

    force(pos, active_mask) -> acc (3, N) for the active particles (others may be anything).
    Returns pos, vel, rung after the last substep (velocities half-kicked as the schedule leaves
    them; call with n_substeps a multiple of 2^R and close() to end on a full step).
    """
    pos = np.array(pos, dtype=np.float64)
    vel = np.array(vel, dtype=np.float64)
    n = pos.shape[1]
    act = np.ones(n, dtype=bool)
    acc = force(pos, act)
    if rung is None:
        rung = target_rungs(acc, eps, dt0, max_rung)
    for k in range(n_substeps):
        s = k % (1 << max_rung)
        pos, vel, rung, act_next = kick_drift(pos, vel, acc, rung, eps, dt0, max_rung, s, closing=(k > 0))
        new = force(pos, act_next)
        acc = np.where(act_next[None, :], new, acc)
        act = act_next
    return pos, vel, rung, acc


def close(vel, acc, rung, dt0):
    """The closing half kick at the end of a base step (all particles are active there)."""
    vel = np.array(vel, dtype=np.float64)
    a = np.asarray(acc, dtype=np.float32).astype(np.float64)
    return vel + a * np.ldexp(dt0, -np.asarray(rung, dtype=np.int64) - 1)


# ---------------------------------------------------------------- compressed storage (Sec. 3.4)
#
# The paper keeps positions as 32-bit integer coordinates of the box and velocities as single
# precision floats.  Reading of the substep on that storage (the same schedule as kick_drift):
#   - a position component is u (uint32), the coordinate u * 2^-32 of the unit box;
#   - the half kicks of a substep run in FP64 from the stored FP32 velocity, v += a hk, each
#     product and each sum rounded once, and the velocity is stored rounded to FP32;
#   - the drift moves u by the nearest integer (ties to even) of (v32 h) 2^32, computed in FP64;
#   - in a periodic box u wraps modulo 2^32; in the isolated box a component that would leave
#     [0, 2^32) leaves the particle where it was and is reported.


def kick_drift_i32(ipos, vel, acc, rung, eps, dt0, max_rung, s, closing, periodic=False):
    """One substep on compressed storage; returns (ipos uint32 (3, N), vel float32 (3, N), rung,
    active_next, out) where out flags the particles an isolated box would lose (left in place)."""
    u = np.array(ipos, dtype=np.uint32).astype(np.int64)
    v = np.asarray(vel, dtype=np.float32).astype(np.float64)
    rung = np.array(rung, dtype=np.int64)
    a = np.asarray(acc, dtype=np.float32).astype(np.float64)
    act = active(rung, s, max_rung)
    if closing:
        v[:, act] = v[:, act] + a[:, act] * np.ldexp(dt0, -rung[act] - 1)
    tgt = target_rungs(acc, eps, dt0, max_rung)
    new = rung.copy()
    for i in np.nonzero(act)[0]:
        rt, r = int(tgt[i]), int(rung[i])
        if rt >= r:
            new[i] = rt
        else:
            rn = rt
            while rn < r and s % (1 << (max_rung - rn)) != 0:
                rn += 1
            new[i] = rn
    rung = new
    v[:, act] = v[:, act] + a[:, act] * np.ldexp(dt0, -rung[act] - 1)
    v32 = np.asarray(vel, dtype=np.float32).copy()
    v32[:, act] = v[:, act].astype(np.float32)
    h = math.ldexp(dt0, -max_rung)
    d = np.rint((v32.astype(np.float64) * h) * 4294967296.0).astype(np.int64)
    un = u + d
    if periodic:
        un &= 0xFFFFFFFF
        out = np.zeros(u.shape[1], dtype=bool)
    else:
        out = np.any((un < 0) | (un > 0xFFFFFFFF), axis=0)
        un[:, out] = u[:, out]
    return un.astype(np.uint32), v32, rung, active(rung, s + 1, max_rung), out


def to_fixed(pos):
    """Nearest 32-bit coordinates of FP64 positions in [0, 1): u = rint(x 2^32), capped at 2^32 - 1."""
    u = np.rint(np.asarray(pos, dtype=np.float64) * 4294967296.0)
    return np.minimum(u, 4294967295.0).astype(np.uint32)


def from_fixed(ipos):
    """The FP64 coordinates u 2^-32 of 32-bit ones (exact)."""
    return np.asarray(ipos, dtype=np.uint32).astype(np.float64) * (1.0 / 4294967296.0)
