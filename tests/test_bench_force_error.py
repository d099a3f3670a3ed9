"""The force-error report of the benchmark line: relative errors against the FP64 direct sum, their
rms, nearest-rank 99th percentile and maximum.  Checked on the CPU with accelerations of known
error, built from the oracle's own direct sum."""
import numpy as np

import bench
import oracle
from paper_1609_08621_gb300 import synth


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
