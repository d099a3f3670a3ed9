"""The force-error report of the benchmark line: relative errors against the FP64 direct sum, their
rms, nearest-rank 99th percentile and maximum.  Checked on the CPU with accelerations of known
error, built from the oracle's own direct sum."""
import numpy as np
import pytest

import bench
import oracle
from paper_1609_08621_gb300 import synth

torch = pytest.importorskip("torch")


def _with_errors(ref, rel, seed=1):
    """ref with a perturbation of relative size rel[i] in a random direction at particle i."""
    d = np.random.default_rng(seed).normal(size=ref.shape)
    d /= np.linalg.norm(d, axis=0)
    return ref + rel * np.linalg.norm(ref, axis=0) * d


def test_force_error_statistics():
    n, eps = 500, 1e-3
    pos, m = synth.clustered_plummer(n, 5)
    ref, _ = oracle.direct(pos, m, eps)
    r = bench.force_error(pos, m, eps, ref, nsinks=n)
    assert r["rms"] < 1e-13 and r["max"] < 1e-13 and r["sinks"] == n
    r = bench.force_error(pos, m, eps, _with_errors(ref, np.full(n, 1e-3)), nsinks=n)
    assert abs(r["rms"] - 1e-3) < 1e-12 and abs(r["p99"] - 1e-3) < 1e-12 and abs(r["max"] - 1e-3) < 1e-12
    # nearest rank: of 500 errors the 99th percentile is the 495th smallest
    rel = np.full(n, 1e-3)
    rel[:5] = 0.1
    assert abs(bench.force_error(pos, m, eps, _with_errors(ref, rel), nsinks=n)["p99"] - 1e-3) < 1e-12
    rel[5] = 0.1
    assert abs(bench.force_error(pos, m, eps, _with_errors(ref, rel), nsinks=n)["p99"] - 0.1) < 1e-12


def test_force_error_samples_distinct_sinks():
    n, eps = 2000, 1e-3
    pos, m = synth.clustered_plummer(n, 6)
    ref, _ = oracle.direct(pos, m, eps)
    rel = np.zeros(n)
    rel[::2] = 1e-2  # half the particles carry an error
    r = bench.force_error(pos, m, eps, _with_errors(ref, rel), nsinks=400)
    assert r["sinks"] == 400
    # a sample of distinct sinks from both halves: rms between the extremes, max at the carried error
    assert 1e-3 < r["rms"] < 1e-2 and abs(r["max"] - 1e-2) < 1e-12


class _ExactCtx:
    """Stands in for the library with exact answers: acc is the oracle's direct sum of the given
    positions (per box for a batch), rounded to FP32.  A correct force_error then reports only that
    rounding; a wrong box, slice or layout reports errors of order one."""

    def compute_forces(self, tpos, tmass, eps, theta, acc, pot=None, active=None):
        a, _ = oracle.direct(tpos.numpy().reshape(3, -1), tmass.numpy(), eps)
        acc.copy_(torch.from_numpy(a.reshape(-1).astype(np.float32)))

    def compute_forces_batch(self, tpos, tmass, off, eps, theta, acc, pot):
        pos, m = tpos.numpy().reshape(3, -1), tmass.numpy()
        out = np.zeros_like(pos)
        for b in range(len(off) - 1):
            sl = slice(int(off[b]), int(off[b + 1]))
            out[:, sl] = oracle.direct(pos[:, sl], m[sl], eps)[0]
        acc.copy_(torch.from_numpy(out.reshape(-1).astype(np.float32)))


def test_workload_force_error_slices_and_layouts():
    from types import SimpleNamespace

    t = torch
    eps = 1e-3
    boxes = [synth.clustered_plummer(n, 20 + n) for n in (300, 900, 500)]
    off = np.concatenate([[0], np.cumsum([b[1].size for b in boxes])])
    pos = np.concatenate([b[0] for b in boxes], axis=1)
    mass = np.concatenate([b[1] for b in boxes])
    n = mass.size
    w = SimpleNamespace(ctx=_ExactCtx(), dev="cpu", pos=pos, mass=mass, boxes=boxes, off=off, n=n, eps=eps,
                        theta=0.7, tmass=t.from_numpy(mass), acc=t.zeros(3 * n, dtype=t.float32),
                        pot=t.zeros(n, dtype=t.float32))
    r = bench.Batch.force_error(w, nsinks=200)
    assert r["box"] == 1 and r["sinks"] == 200 and r["max"] < 1e-6
    one = SimpleNamespace(ctx=_ExactCtx(), dev="cpu", pos=boxes[0][0], mass=boxes[0][1], n=300, eps=eps,
                          theta=0.7, tmass=t.from_numpy(boxes[0][1]), acc=t.zeros(900, dtype=t.float32))
    for cls in (bench.Box, bench.Rungs):
        r = cls.force_error(one, nsinks=100)
        assert r["sinks"] == 100 and r["max"] < 1e-6
