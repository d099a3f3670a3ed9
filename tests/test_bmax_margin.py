"""The FP32 error margin behind the exact b_max (Sec. 3.1, b_max = distance from the centre of mass to
the farthest particle), checked on the CPU.

The upward pass and the b_max passes evaluate the exact FP64 distance only for particles whose FP32
distance from the FP32-rounded centre reaches (largest FP32 distance) - (4e-7 + 6e-7 d).  That keeps
the farthest particle among the candidates if every FP32 distance is within half that margin of the
exact one, i.e. |d32 - d| <= 2e-7 + 3e-7 d; the kernels' comments state the tighter
1.1e-7 + 1.3e-7 d for positions in [0, 1).  Here d32 is formed exactly as the kernels form it:
rounded coordinates and centre, one FP32 subtraction per axis, ((dx dx) + dy dy) + dz dz with the
last two steps fused, and a correctly rounded square root.
"""
import numpy as np

f32 = np.float32


def _fma32(a, b, c):
    """fl32(a b + c): the float product is exact in FP64, and for these magnitudes the FP64 sum
    rounds to the same float as the exact one."""
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(f32)


def _d32(x, c):
    """The kernels' FP32 distance between positions x (n, 3) and centre c (n, 3), both FP64."""
    xs, cs = x.astype(f32), c.astype(f32)
    d = (xs - cs).astype(f32)
    dx, dy, dz = d[:, 0], d[:, 1], d[:, 2]
    s = _fma32(dz, dz, _fma32(dy, dy, (dx * dx).astype(f32)))
    return np.sqrt(s.astype(f32)).astype(f32)


def _cases(rng, n):
    # centres anywhere in the box, with extra weight near 1 where the float spacing is largest
    c = rng.random((n, 3))
    c[: n // 4] = 1.0 - rng.random((n // 4, 3)) * 1e-3
    c[n // 4: n // 2] = rng.random((n // 4, 3)) * 1e-6
    # offsets from 1e-9 to 0.5 of the box, random directions, positions kept in [0, 1)
    r = 10.0 ** rng.uniform(-9, np.log10(0.5), n)
    u = rng.normal(size=(n, 3))
    u /= np.linalg.norm(u, axis=1)[:, None]
    x = np.clip(c + r[:, None] * u, 0.0, np.nextafter(1.0, 0.0))
    return x, c


def test_fp32_distance_within_the_stated_bound():
    rng = np.random.default_rng(11)
    x, c = _cases(rng, 400000)
    d = np.linalg.norm(x - c, axis=1)
    err = np.abs(_d32(x, c).astype(np.float64) - d)
    assert np.all(err <= 1.1e-7 + 1.3e-7 * d), float(np.max(err - (1.1e-7 + 1.3e-7 * d)))


def test_margin_keeps_the_farthest_particle():
    """Clusters around a centre of mass: the particle with the largest exact distance always passes
    the candidate test, while most particles do not (the test saves FP64 work)."""
    rng = np.random.default_rng(12)
    kept, total = 0, 0
    for trial in range(300):
        n = int(rng.integers(2, 2048))
        scale = 10.0 ** rng.uniform(-7, -0.5)
        c0 = rng.random(3) * (1 - 2 * scale) + scale
        x = np.clip(c0 + scale * rng.normal(size=(n, 3)) / 3, 0.0, np.nextafter(1.0, 0.0))
        com = x.mean(axis=0)
        cc = np.broadcast_to(com, x.shape)
        d = np.linalg.norm(x - cc, axis=1)
        d32 = _d32(x, cc)
        top = f32(np.max(d32))  # the square root of the largest square: the same value
        thr = f32(top - f32(f32(4e-7) + f32(f32(6e-7) * top)))
        cand = d32 >= thr
        assert cand[np.argmax(d)], trial
        kept += int(cand.sum())
        total += n
    assert kept < 0.2 * total
