"""Several isolated boxes in one solve (fmm_compute_forces_batch): every box's forces are the
same as solving that box alone -- bit for bit, since its subtree, lists and arithmetic are the
same -- and agree with the oracle FMM of that box alone."""
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


def t(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a).reshape(-1)).to("cuda:0", dtype)


def solve_batch(ctx, boxes, eps, theta):
    pos = np.concatenate([b[0] for b in boxes], axis=1)
    mass = np.concatenate([b[1] for b in boxes])
    off = np.zeros(len(boxes) + 1, np.int64)
    off[1:] = np.cumsum([b[1].size for b in boxes])
    n = mass.size
    acc = torch.full((3 * n,), float("nan"), dtype=torch.float32, device="cuda:0")
    pot = torch.full((n,), float("nan"), dtype=torch.float32, device="cuda:0")
    ctx.compute_forces_batch(t(pos, torch.float64), t(mass, torch.float32), off, eps, theta, acc, pot)
    torch.cuda.synchronize()
    return acc.cpu().numpy().reshape(3, n), pot.cpu().numpy(), off


def solve_one(ctx, pos, mass, eps, theta):
    n = mass.size
    acc = torch.zeros(3 * n, dtype=torch.float32, device="cuda:0")
    pot = torch.zeros(n, dtype=torch.float32, device="cuda:0")
    ctx.compute_forces(t(pos, torch.float64), t(mass, torch.float32), eps, theta, acc, pot)
    torch.cuda.synchronize()
    return acc.cpu().numpy().reshape(3, n), pot.cpu().numpy()


def test_batch_equals_single_boxes_bitwise(ctx):
    sizes = [5000, 1, 17, 12345, 64, 3000, 65]
    boxes = [synth.clustered_plummer(k, 100 + i) for i, k in enumerate(sizes)]
    acc, pot, off = solve_batch(ctx, boxes, 1e-3, 0.7)
    for b, (p, m) in enumerate(boxes):
        a1, p1 = solve_one(ctx, p, m, 1e-3, 0.7)
        sl = slice(off[b], off[b + 1])
        assert np.array_equal(acc[:, sl], a1) and np.array_equal(pot[sl], p1), b


def test_batch_matches_oracle_per_box(ctx):
    boxes = [synth.clustered_plummer(k, 200 + i) for i, k in enumerate([9000, 4096, 20000])]
    acc, pot, off = solve_batch(ctx, boxes, 1e-3, 0.7)
    for b, (p, m) in enumerate(boxes):
        ra, rp = oracle.FMM(p, m, 1e-3, 0.7).forces()
        ref, _ = oracle.direct(p, m, 1e-3)
        a = acc[:, off[b]:off[b + 1]].astype(np.float64)
        e = np.linalg.norm(a - ra, axis=0) / np.linalg.norm(ref, axis=0)
        assert e.max() <= 2e-3 and np.sqrt(np.mean(e ** 2)) <= 2e-5
        et = np.linalg.norm(a - ref, axis=0) / np.linalg.norm(ref, axis=0)
        assert np.sqrt(np.mean(et ** 2)) <= 1e-3


def test_batch_with_empty_boxes_and_bad_offsets(ctx):
    boxes = [synth.clustered_plummer(k, 300 + i) for i, k in enumerate([2000, 3000])]
    pos = np.concatenate([b[0] for b in boxes], axis=1)
    mass = np.concatenate([b[1] for b in boxes])
    n = mass.size
    acc = torch.zeros(3 * n, dtype=torch.float32, device="cuda:0")
    off = np.array([0, 0, 2000, 2000, n], np.int64)
    ctx.compute_forces_batch(t(pos, torch.float64), t(mass, torch.float32), off, 1e-3, 0.7, acc)
    a = acc.cpu().numpy().reshape(3, n)
    a0, _ = solve_one(ctx, boxes[0][0], boxes[0][1], 1e-3, 0.7)
    assert np.array_equal(a[:, :2000], a0)
    for bad in ([0, 10, 5, n], [1, n], [0, n - 1]):
        with pytest.raises(binding.FmmError):
            ctx.compute_forces_batch(t(pos, torch.float64), t(mass, torch.float32), np.array(bad, np.int64), 1e-3,
                                     0.7, acc)
