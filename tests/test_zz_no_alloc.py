"""The allocation-free Morton order (fmm_morton_order_static) against the context path
(fmm_build_tree, then fmm_export_order) and the oracle's own keys and order: identical keys and
order on two calls in a row, the size limit of its fixed scratch, invalid positions, and no
device allocation after the first call.  Collected last on purpose, so that it runs both alone
and after every other test in one process."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1609_08621_gb300 import binding, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _context_order(pos, mass, dev):
    ctx = binding.Context(0)
    try:
        ctx.build_tree(torch.from_numpy(pos.reshape(-1)).to(dev), torch.from_numpy(mass).to(dev))
        return ctx.export_order(mass.size)
    finally:
        ctx.close()


def _static_order(pos_dev, keys, order):
    binding.morton_order_static(pos_dev, keys, order)
    return order.cpu().numpy().view(np.uint32).copy(), keys.cpu().numpy().view(np.uint64).copy()


def test_two_calls_match_the_context_path(dev):
    # a clustered set spanning many sort tiles with a ragged tail, then a set of coincident
    # particles where every key ties and the order must stay the input order
    pa, ma = synth.clustered_plummer(300001, 11)
    pb, mb = synth.coincident(70003, 12, n_points=3)
    bufs = []
    for p in (pa, pb):
        n = p.shape[1]
        bufs.append((torch.from_numpy(np.ascontiguousarray(p).reshape(-1)).to(dev),
                     torch.empty(n, dtype=torch.int64, device=dev), torch.empty(n, dtype=torch.int32, device=dev)))
    torch.cuda.synchronize()
    got_a = _static_order(*bufs[0])
    got_b = _static_order(*bufs[1])
    ref_a = _context_order(pa, ma, dev)
    ref_b = _context_order(pb, mb, dev)
    for got, ref in ((got_a, ref_a), (got_b, ref_b)):
        assert np.array_equal(got[0], ref[0])
        assert np.array_equal(got[1], ref[1])
    # the oracle's Morton keys and order (Sec. 3.1, its own quantisation and sort), with no
    # active sink so that its walk does no work
    for got, (p, m) in ((got_a, (pa, ma)), (got_b, (pb, mb))):
        orc = oracle.FMM(p, m, 1e-3, 0.7, active=np.zeros(m.size, np.uint8))
        assert np.array_equal(got[0].astype(np.int64), orc.perm())
        assert np.array_equal(got[1], orc.keys())
    assert np.all(np.diff(got_a[1].astype(np.float64)) >= 0)
    # equal keys keep the input order
    same = np.diff(got_b[1]) == 0
    assert np.all(np.diff(got_b[0].astype(np.int64))[same] > 0)


def test_limit_and_invalid_positions(dev):
    m = binding.STATIC_ORDER_MAX_N
    over = m + 1
    with pytest.raises(binding.FmmError) as e:
        binding.morton_order_static(torch.zeros(3 * over, dtype=torch.float64, device=dev),
                                    torch.empty(over, dtype=torch.int64, device=dev),
                                    torch.empty(over, dtype=torch.int32, device=dev))
    assert "outside" in str(e.value)
    # the largest size is accepted and still matches the context path
    p, ms = synth.clustered_plummer(m, 13)
    keys = torch.empty(m, dtype=torch.int64, device=dev)
    order = torch.empty(m, dtype=torch.int32, device=dev)
    got = _static_order(torch.from_numpy(np.ascontiguousarray(p).reshape(-1)).to(dev), keys, order)
    ref = _context_order(p, ms, dev)
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])
    # a position outside the unit box is reported, and the next call works again
    bad = np.ascontiguousarray(p[:, :1000]).copy()
    bad[1, 17] = 1.0
    with pytest.raises(binding.FmmError):
        binding.morton_order_static(torch.from_numpy(bad.reshape(-1)).to(dev), keys[:1000], order[:1000])
    good = np.ascontiguousarray(p[:, :1000])
    got = _static_order(torch.from_numpy(good.reshape(-1)).to(dev), keys[:1000], order[:1000])
    ref = _context_order(good, np.ascontiguousarray(ms[:1000]), dev)
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])


def test_no_device_allocation_after_the_first_call(dev):
    # after one call has set the device up, calls at the largest size change neither the
    # device's free memory nor the torch allocator's counters: the scratch is the library's
    # fixed array, and the caller's buffers are all that the call writes
    m = binding.STATIC_ORDER_MAX_N
    p, _ = synth.clustered_plummer(m, 14)
    pos = torch.from_numpy(np.ascontiguousarray(p).reshape(-1)).to(dev)
    keys = torch.empty(m, dtype=torch.int64, device=dev)
    order = torch.empty(m, dtype=torch.int32, device=dev)
    binding.morton_order_static(pos, keys, order)
    torch.cuda.synchronize()
    first = order.cpu()
    free0, _ = torch.cuda.mem_get_info(dev)
    stats0 = torch.cuda.memory_stats(dev)
    for _ in range(4):
        binding.morton_order_static(pos, keys, order)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info(dev)
    stats1 = torch.cuda.memory_stats(dev)
    assert free1 == free0
    for k in ("allocation.all.allocated", "segment.all.allocated", "reserved_bytes.all.current"):
        assert stats1.get(k, 0) == stats0.get(k, 0), k
    assert torch.equal(order.cpu(), first)
