"""The values the paper prints (tests/golden/paper_parameters.txt, each with its citation) against
the ones the library, the generated operators and the oracle use."""
import os
import re

import numpy as np
import pytest

import oracle
from oracle import kdk
from paper_1609_08621_gb300 import binding, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _n_indices(order):
    """Multi-indices n of three components with |n| <= order."""
    return sum(1 for a in range(order + 1) for b in range(order + 1 - a) for _ in range(order + 1 - a - b))


def test_library_defaults_are_the_papers(paper):
    p = binding.fmm_default_params()  # host only: fills the struct, no device call
    assert p.bucket == paper["bucket_size"] and p.group == paper["group_size"]
    assert p.group == 4 * p.bucket  # "four times the bucket size"
    assert p.theta == paper["theta_mid"]


def test_expansion_orders(paper):
    lo, mo = int(paper["local_order"]), int(paper["multipole_order"])
    assert oracle.NMI == _n_indices(lo) and oracle.NM4 == _n_indices(mo)
    hdr = open(os.path.join(ROOT, "paper_1609_08621_gb300", "csrc", "expansions.cuh")).read()
    assert int(re.search(r"#define FMM_NL (\d+)", hdr).group(1)) == _n_indices(lo)
    # moments about the centre of mass: the dipole vanishes and is not stored
    assert int(re.search(r"#define FMM_NMOM (\d+)", hdr).group(1)) == _n_indices(mo) - 3
    loc, mom = binding.fmm_multi_index()
    assert loc.sum(axis=1).max() == lo and mom.sum(axis=1).max() == mo


def test_softening_rule(paper):
    for n in (4096, 128 ** 3, 256 ** 3, 512 ** 3):
        assert synth.paper_softening(n) == pytest.approx(paper["softening_per_sep"] / n ** (1.0 / 3.0), rel=1e-15)


def test_timestep_rule(paper):
    rng = np.random.default_rng(3)
    acc = rng.normal(size=(3, 64)).astype(np.float32)
    eps = 1e-3
    want = paper["timestep_eta"] * np.sqrt(eps / np.linalg.norm(acc.astype(np.float64), axis=0))
    assert np.allclose(kdk.timestep(acc, eps), want, rtol=1e-12)


def test_workload_opening_angles_are_the_papers(paper):
    thetas = {paper["theta_early"], paper["theta_mid"], paper["theta_late"]}
    for name, w in synth.WORKLOADS.items():
        if "theta" in w:
            assert w["theta"] in thetas, name
