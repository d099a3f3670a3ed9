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
