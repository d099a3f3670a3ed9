"""Parity of the CUDA path with the CPU oracle, stage by stage, through the C ABI.

Tolerances (derived from the arithmetic):
* integer and index work (sort order, keys, tree topology, interaction lists): exact;
* FP64 tree geometry (mass, centre of mass, b_max): the two sides sum in different orders,
  so 1e-12 relative; bounding boxes are min/max and therefore exact;
* FP32 moments: each is a sum of <= count terms m y^n of one sign structure, formed from
  offsets rounded to FP32 (relative 2^-24) and shifted by M2M in FP32, so |dM_n| <= 1e-5 of the
  cell's scale m b_max^|n|;
* FP32 forces against the FP64 oracle FMM on identical lists: every term carries a few units
  of 2^-24 relative error and the sums cancel by a factor kappa = sum|terms| / |a| (tens for
  clustered sets), so per-particle errors are ~1e-6..1e-5 of |a|: rms <= 2e-5, max <= 2e-3;
* against the FP64 direct sum: the method's own truncation error, rms <= 1e-3 and
  99th percentile <= 1e-2 (the target accuracy of the solve).
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1609_08621_gb300 import binding, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = binding.Context(0)
    yield c
    c.close()


def dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a).reshape(-1)).to("cuda:0", dtype)


def gpu_solve(ctx, pos, mass, eps, theta, active=None, terms=7, bucket=16, group=64):
    n = mass.size
    ctx.set_params(terms=terms, bucket=bucket, group=group)
    acc = torch.full((3 * n,), float("nan"), dtype=torch.float32, device="cuda:0")
    pot = torch.full((n,), float("nan"), dtype=torch.float32, device="cuda:0")
    act = None if active is None else dev(active, torch.uint8)
    ctx.compute_forces(dev(pos, torch.float64), dev(mass, torch.float32), eps, theta, acc, pot, act)
    torch.cuda.synchronize()
    ctx.set_params(terms=7, bucket=16, group=64)
    return acc.cpu().numpy().reshape(3, n).astype(np.float64), pot.cpu().numpy().astype(np.float64)


def rel_err(a, ref):
    return np.linalg.norm(a - ref, axis=0) / np.linalg.norm(ref, axis=0)


def rms(x):
    return float(np.sqrt(np.mean(np.square(x))))


# ---------------------------------------------------------------- tree


@pytest.mark.parametrize("kind,n,seed", [("plummer", 20000, 3), ("nfw", 30011, 4), ("coincident", 3000, 5)])
def test_tree_matches_oracle(ctx, kind, n, seed):
    pos, mass = synth.make(kind, n, seed)
    ctx.build_tree(dev(pos, torch.float64), dev(mass, torch.float32))
    perm, keys = ctx.export_order(n)
    orc = oracle.FMM(pos, mass, 1e-3, 0.7)
    assert np.array_equal(perm.astype(np.int64), orc.perm())
    assert np.array_equal(keys, orc.keys())
    g = ctx.export_cells()
    o = orc.cells()
    gk = {(int(f), int(c)): i for i, (f, c) in enumerate(zip(g["first"], g["count"]))}
    ok = {(int(f), int(c)): i for i, (f, c) in enumerate(zip(o["first"], o["count"]))}
    assert gk.keys() == ok.keys()
    gi = np.array([gk[k] for k in ok])
    oi = np.array(list(ok.values()))

    def rng(d, i):
        return (int(d["first"][i]), int(d["count"][i])) if i >= 0 else None

    for a, b in zip(gi, oi):
        assert rng(g, g["parent"][a]) == rng(o, o["parent"][b])
        assert [rng(g, x) for x in g["child"][a]] == [rng(o, x) for x in o["child"][b]]
    assert np.allclose(g["mass"][gi], o["mass"][oi], rtol=1e-12)
    assert np.allclose(g["com"][gi], o["com"][oi], rtol=1e-12, atol=1e-15)
    assert np.array_equal(g["lo"][gi], o["lo"][oi]) and np.array_equal(g["hi"][gi], o["hi"][oi])
    # b_max is exact given the centre of mass, which both sides sum in different orders:
    # an absolute difference of a few FP64 ulps of the unit box (<= N * 2^-53) is rounding
    assert np.allclose(g["bmax"][gi], o["bmax"][oi], rtol=1e-12, atol=n * 2.0 ** -52)
    assert np.array_equal(g["nact"][gi], o["nact"][oi])
    # moments: GPU slots are multi-indices of order 0, 2, 3, 4; oracle stores all |n| <= 4
    _, mom_idx = binding.fmm_multi_index()
    mi = oracle.multi_index()
    col = [int(np.where((mi == m).all(axis=1))[0][0]) for m in mom_idx]
    order = mom_idx.sum(axis=1)
    gm = g["moments"][gi][:, :32].astype(np.float64)
    om = o["mom"][oi][:, col]
    # FP32 rounding of each moment (1e-5 of m b^n) plus the noise of the centre of mass itself:
    # the two sides' centres differ by up to delta = N FP64 ulps of the unit box, which moves
    # every offset by delta and a moment by at most M ((b + delta)^n - b^n)
    b = o["bmax"][oi][:, None]
    M = o["mass"][oi][:, None]
    delta = n * 2.0 ** -52
    tol = 1e-5 * M * b ** order[None, :] + 2.0 * M * ((b + delta) ** order[None, :] - b ** order[None, :])
    assert np.all(np.abs(gm - om) <= tol + 1e-30)


# ---------------------------------------------------------------- lists


def _set_of(sink_rng, first, count):
    return set(zip(map(tuple, sink_rng), first.tolist(), count.tolist()))


@pytest.mark.parametrize("kind,n,theta", [("plummer", 20000, 0.7), ("nfw", 20000, 0.55), ("uniform", 9000, 0.4)])
def test_interaction_lists_match_oracle(ctx, kind, n, theta):
    pos, mass = synth.make(kind, n, 7)
    eps = synth.paper_softening(n)
    gpu_solve(ctx, pos, mass, eps, theta)
    g = ctx.export_cells()
    orc = oracle.FMM(pos, mass, eps, theta)
    o = orc.cells()
    grng = np.stack([g["first"], g["count"]], axis=1)
    orng = np.stack([o["first"], o["count"]], axis=1)
    for kind_ in ("pp", "pc", "cc", "cp"):
        s, f, c = ctx.export_lists(kind_)
        os_, of, oc = orc.entries(kind_)
        gs = _set_of(grng[s], f, c)
        ost = _set_of(orng[os_], of, oc)
        assert len(gs) == len(s) and len(ost) == len(os_)
        assert gs == ost, f"{kind_}: gpu-only {len(gs - ost)}, oracle-only {len(ost - gs)}"


# ---------------------------------------------------------------- forces


@pytest.mark.parametrize("kind,n,theta", [("plummer", 12000, 0.7), ("nfw", 16384, 0.55)])
def test_forces_match_oracle_fmm_term_by_term(ctx, kind, n, theta):
    pos, mass = synth.make(kind, n, 9)
    eps = synth.paper_softening(n)
    orc = oracle.FMM(pos, mass, eps, theta)
    tot, _ = orc.forces(7)
    scale = np.linalg.norm(tot, axis=0)
    for terms in (1, 2, 4, 7):
        a, p = gpu_solve(ctx, pos, mass, eps, theta, terms=terms)
        ra, rp = orc.forces(terms)
        e = np.linalg.norm(a - ra, axis=0) / scale
        assert rms(e) <= 2e-5 and e.max() <= 2e-3, (terms, rms(e), e.max())
        ep = np.abs(p - rp) / np.abs(orc.forces(7)[1])
        assert rms(ep) <= 2e-5, (terms, rms(ep))


def test_small_config_against_direct_sum(ctx):
    n, eps, theta = 4096, 1e-3, 0.7
    pos, mass = synth.clustered_plummer(n, 1)
    a, p = gpu_solve(ctx, pos, mass, eps, theta)
    ref, rp = oracle.direct(pos, mass, eps)
    e = rel_err(a, ref)
    assert rms(e) <= 1e-3 and np.quantile(e, 0.99) <= 1e-2
    assert rms((p - rp) / rp) <= 1e-3


def test_full_size_nfw_sampled_against_direct_sum(ctx):
    """The 128^3 NFW workload at full size; 2048 random sinks checked against the FP64 direct sum."""
    n = 128 ** 3
    pos, mass = synth.clustered_nfw(n, 2)
    eps, theta = synth.paper_softening(n), 0.55
    a, p = gpu_solve(ctx, pos, mass, eps, theta)
    assert np.all(np.isfinite(a)) and np.all(np.isfinite(p))
    sinks = np.random.default_rng(0).choice(n, 2048, replace=False)
    ref, rp = oracle.direct(pos, mass, eps, sinks)
    e = rel_err(a[:, sinks], ref)
    assert rms(e) <= 1e-3 and np.quantile(e, 0.99) <= 1e-2, (rms(e), np.quantile(e, 0.99))
    st = ctx.stats()
    assert st["n_pp_pairs"] > 0 and st["n_pc_pairs"] > 0 and st["n_cc"] > 0


# ---------------------------------------------------------------- edge cases


@pytest.mark.parametrize("n", [1, 2, 3, 17, 64, 65, 1000])
def test_tiny_and_ragged_sizes(ctx, n):
    pos, mass = synth.clustered_plummer(n, 40 + n)
    a, p = gpu_solve(ctx, pos, mass, 1e-3, 0.7)
    ref, rp = oracle.direct(pos, mass, 1e-3)
    if n == 1:
        assert np.all(a == 0) and p[0] == 0
        return
    ra, _ = oracle.FMM(pos, mass, 1e-3, 0.7).forces()
    e = np.linalg.norm(a - ra, axis=0) / np.linalg.norm(ref, axis=0)
    assert e.max() <= 2e-3
    assert rms(rel_err(a, ref)) <= 1e-3


def test_coincident_points(ctx):
    pos, mass = synth.coincident(500, 8, n_points=5)
    a, p = gpu_solve(ctx, pos, mass, 1e-3, 0.3)
    ra, rp = oracle.FMM(pos, mass, 1e-3, 0.3).forces()
    e = np.linalg.norm(a - ra, axis=0) / np.linalg.norm(ra, axis=0)
    assert e.max() <= 1e-4
    # all particles at one point: the force vanishes, every potential is -(M - m)/eps
    pos1, mass1 = synth.coincident(300, 9, n_points=1)
    a1, p1 = gpu_solve(ctx, pos1, mass1, 1e-3, 0.7)
    assert np.all(np.abs(a1) <= 1e-3)
    assert np.allclose(p1, -(1.0 - 1.0 / 300) / 1e-3, rtol=1e-5)


def test_active_subset_matches_full_solve(ctx):
    n = 20000
    pos, mass = synth.clustered_plummer(n, 12)
    act = (np.random.default_rng(1).random(n) < 0.1).astype(np.uint8)
    full, fp = gpu_solve(ctx, pos, mass, 1e-3, 0.7)
    part, pp = gpu_solve(ctx, pos, mass, 1e-3, 0.7, active=act)
    sel = act.astype(bool)
    # the same interaction lists; only the split of each sink's sums across lanes follows the
    # group's active count, so the results agree to FP32 summation order
    na = np.linalg.norm(full[:, sel], axis=0)
    assert np.all(np.linalg.norm(part[:, sel] - full[:, sel], axis=0) <= 2e-6 * na)
    assert np.all(np.abs(pp[sel] - fp[sel]) <= 2e-6 * np.abs(fp[sel]))
    assert np.all(np.isnan(part[:, ~sel]))
    assert ctx.stats()["n_active"] == int(sel.sum())
    none, _ = gpu_solve(ctx, pos, mass, 1e-3, 0.7, active=np.zeros(n, np.uint8))
    assert np.all(np.isnan(none))


def test_deterministic_and_host_entry_point(ctx):
    n = 30000
    pos, mass = synth.clustered_nfw(n, 13)
    a1, p1 = gpu_solve(ctx, pos, mass, 2e-4, 0.55)
    a2, p2 = gpu_solve(ctx, pos, mass, 2e-4, 0.55)
    assert np.array_equal(a1, a2) and np.array_equal(p1, p2)
    acc = np.zeros(3 * n, np.float32)
    pot = np.zeros(n, np.float32)
    ctx.compute_forces_host(np.ascontiguousarray(pos.reshape(-1)), mass, 2e-4, 0.55, acc, pot)
    assert np.array_equal(acc.reshape(3, n).astype(np.float64), a1) and np.array_equal(pot.astype(np.float64), p1)


def test_invalid_inputs_are_rejected(ctx):
    n = 100
    pos, mass = synth.uniform_box(n, 3)
    bad = pos.copy()
    bad[1, 7] = 1.0
    acc = torch.zeros(3 * n, dtype=torch.float32, device="cuda:0")
    with pytest.raises(binding.FmmError) as ei:
        ctx.compute_forces(dev(bad, torch.float64), dev(mass, torch.float32), 1e-3, 0.7, acc)
    assert ei.value.status == -1
    for eps, theta in ((0.0, 0.7), (1e-3, 0.0), (1e-3, 1.5), (float("nan"), 0.7)):
        with pytest.raises(binding.FmmError):
            ctx.compute_forces(dev(pos, torch.float64), dev(mass, torch.float32), eps, theta, acc)
    m2 = mass.copy()
    m2[3] = 0.0
    with pytest.raises(binding.FmmError):
        ctx.compute_forces(dev(pos, torch.float64), dev(m2, torch.float32), 1e-3, 0.7, acc)
    # the context stays usable
    a, _ = gpu_solve(ctx, pos, mass, 1e-3, 0.7)
    assert np.all(np.isfinite(a))


def test_group_and_bucket_sizes(ctx):
    n = 8000
    pos, mass = synth.clustered_plummer(n, 14)
    ref, _ = oracle.direct(pos, mass, 1e-3)
    for b, g in ((1, 1), (4, 16), (8, 32), (16, 16), (16, 64)):
        a, _ = gpu_solve(ctx, pos, mass, 1e-3, 0.55, bucket=b, group=g)
        ra, _ = oracle.FMM(pos, mass, 1e-3, 0.55, bucket=b, group=g).forces()
        e = np.linalg.norm(a - ra, axis=0) / np.linalg.norm(ref, axis=0)
        assert e.max() <= 2e-3 and rms(e) <= 2e-5, (b, g, e.max())


def test_fp64_combine_option(ctx):
    """accumulate = 1 adds a particle's chunk partial sums and local-expansion term in FP64: the
    result stays within FP32 rounding of the FP32 combine, and no further from the oracle FMM."""
    n, eps, theta = 30000, synth.paper_softening(30000), 0.55
    pos, mass = synth.clustered_nfw(n, 21)
    a0, p0 = gpu_solve(ctx, pos, mass, eps, theta)
    ctx.set_params(accumulate=1)
    try:
        a1, p1 = gpu_solve(ctx, pos, mass, eps, theta)
    finally:
        ctx.set_params(accumulate=0)
    ra, rp = oracle.FMM(pos, mass, eps, theta).forces()
    scale = np.linalg.norm(ra, axis=0)
    e0 = np.linalg.norm(a0 - ra, axis=0) / scale
    e1 = np.linalg.norm(a1 - ra, axis=0) / scale
    assert rms(np.linalg.norm(a1 - a0, axis=0) / scale) <= 1e-5
    assert rms(e1) <= 1.05 * rms(e0) + 1e-7 and e1.max() <= 2e-3
    assert rms((p1 - rp) / rp) <= 1e-5
    with pytest.raises(binding.FmmError):
        ctx.set_params(accumulate=2)


def test_tight_theta_reference_against_direct_sum(ctx):
    """The error reference of the learned-criterion benchmark -- an FMM solve at theta = 0.25 with
    the FP64 combine, restricted to the sampled sinks -- against the FP64 direct sum, on the
    full-size 128^3 NFW box: its own error must be far below the 1e-4 errors it measures."""
    n = 128 ** 3
    pos, mass = synth.clustered_nfw(n, 2)
    eps = synth.paper_softening(n)
    sinks = np.sort(np.random.default_rng(1).choice(n, 2048, replace=False))
    act = np.zeros(n, np.uint8)
    act[sinks] = 1
    ctx.set_params(accumulate=1)
    try:
        a, _ = gpu_solve(ctx, pos, mass, eps, 0.25, active=act)
    finally:
        ctx.set_params(accumulate=0)
    ref, _ = oracle.direct(pos, mass, eps, sinks)
    e = rel_err(a[:, sinks], ref)
    print(f"\nreference theta=0.25: rms {rms(e):.3e} max {e.max():.3e}")
    # measured: rms 9.7e-7, max 7.0e-6
    assert rms(e) <= 3e-6 and e.max() <= 3e-5, (rms(e), e.max())


def test_list_chunk_sizes(ctx):
    """The work-item size only regroups each sink's partial sums: same interaction counts, forces
    equal to FP32 rounding, for chunks of 32, 64 (default) and 128 entries."""
    n, eps, theta = 20000, 1e-3, 0.55
    pos, mass = synth.clustered_plummer(n, 31)
    res = {}
    for ch in (32, 64, 128):
        ctx.set_params(list_chunk=ch)
        try:
            a, _ = gpu_solve(ctx, pos, mass, eps, theta)
        finally:
            ctx.set_params(list_chunk=0)
        st = ctx.stats()
        res[ch] = (a, st["n_pp_pairs"], st["n_pc_pairs"])
    a64 = res[64][0]
    for ch in (32, 128):
        assert res[ch][1:] == res[64][1:]
        assert rms(np.linalg.norm(res[ch][0] - a64, axis=0) / np.linalg.norm(a64, axis=0)) <= 1e-6
    for bad in (16, 48, 2048):
        with pytest.raises(binding.FmmError):
            ctx.set_params(list_chunk=bad)


def test_autotune_picks_a_candidate(ctx):
    n, eps, theta = 60000, 1e-3, 0.55
    pos, mass = synth.clustered_plummer(n, 32)
    tp, tm = dev(pos, torch.float64), dev(mass, torch.float32)
    acc = torch.zeros(3 * n, dtype=torch.float32, device="cuda:0")
    cands = [(16, 64, 64), (8, 32, 32), (12, 48, 128)]
    best, ms = ctx.autotune(tp, tm, eps, theta, acc, candidates=cands, reps=1)
    assert (best.bucket, best.group, best.list_chunk) in cands and ms > 0
    p = ctx.get_params()
    assert (p.bucket, p.group, p.list_chunk) == (best.bucket, best.group, best.list_chunk)
    # the tuned context still solves correctly
    a, _ = gpu_solve(ctx, pos, mass, eps, theta, bucket=best.bucket, group=best.group)
    ref, _ = oracle.direct(pos, mass, eps, np.arange(0, n, 97))
    e = rel_err(a[:, ::97], ref)
    assert rms(e) <= 1e-3 and np.quantile(e, 0.99) <= 1e-2
    # an invalid candidate is an error and leaves the parameters as they were
    p = ctx.get_params()
    with pytest.raises(binding.FmmError):
        ctx.autotune(tp, tm, eps, theta, acc, candidates=[(16, 64, 48)], reps=1)
    p2 = ctx.get_params()
    assert (p2.bucket, p2.group, p2.list_chunk) == (p.bucket, p.group, p.list_chunk)
    ctx.set_params(bucket=16, group=64, list_chunk=0)
