"""The integer forms of the FP64 conversions the tree kernels use (csrc/f64bits.cuh), compiled for the
host with g++ and compared bit for bit with the host's own IEEE-754 operations.

The kernels replace FP64 instructions (1/64 of the FP32 issue rate on the GPU) by integer work on
the encodings: the range check 0 <= x < 1, the Morton quantisation floor(x 2^21), the rounding of
a double to single precision, and the float pair (fl(x), fl(x - fl(x))) that carries a position or
centre.  Each must equal the plain operation exactly, since keys, tree and centres feed the exact
list parity.  Inputs: every binade from 2^-1100 to 2^130 (both signs), values at and next to the
rounding ties, the boundaries of the fast paths, zeros, infinities and NaN.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1609_08621_gb300", "csrc")

HARNESS = r"""
#define __host__
#define __device__
#define __forceinline__ inline
#include "f64bits.cuh"
extern "C" {
void h_convert(const double* x, long long n, float* f, float* h, float* l, unsigned int* q, unsigned char* in) {
    for (long long i = 0; i < n; i++) {
        f[i] = fmm_d2f_rn(x[i]);
        fmm_split_f32(x[i], h[i], l[i]);
        q[i] = fmm_quantise21(x[i]);
        in[i] = fmm_in_unit(x[i]) ? 1 : 0;
    }
}
void h_widen(const float* f, long long n, double* d) {
    for (long long i = 0; i < n; i++) d[i] = fmm_f2d(f[i]);
}
void h_keys(const double* x, long long n, unsigned long long* k, double* back) {
    for (long long i = 0; i < n; i++) { k[i] = fmm_nonneg_key(x[i]); back[i] = fmm_dfrom(k[i]); }
}
}
"""


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("f64bits")
    src = d / "h.cpp"
    src.write_text(HARNESS)
    so = d / "libh.so"
    subprocess.run(["g++", "-O2", "-fno-fast-math", "-ffp-contract=off", "-shared", "-fPIC", f"-I{CSRC}",
                    str(src), "-o", str(so)], check=True)
    L = ctypes.CDLL(str(so))
    L.h_convert.restype = None
    L.h_widen.restype = None
    L.h_keys.restype = None
    return L


def run(lib, x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    n = x.size
    f = np.empty(n, np.float32)
    h = np.empty(n, np.float32)
    l = np.empty(n, np.float32)
    q = np.empty(n, np.uint32)
    i = np.empty(n, np.uint8)
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    lib.h_convert(p(x), ctypes.c_longlong(n), p(f), p(h), p(l), p(q), p(i))
    return f, h, l, q, i.astype(bool)


def inputs():
    rng = np.random.default_rng(7)
    parts = []
    # random significands in every binade, both signs
    e = np.arange(-1100, 131)
    m = rng.random((e.size, 64)) + 1.0
    v = (m * np.exp2(e.astype(np.float64))[:, None]).ravel()
    parts += [v, -v]
    # uniform in [0, 1), the positions' range
    parts.append(rng.random(200000))
    # exact ties and their neighbours for the float rounding (29 dropped bits 0x10000000) and for
    # the second rounding of the low part
    base = rng.random(20000) + 1.0
    bits = base.view(np.uint64) & ~np.uint64((1 << 29) - 1)
    for off in (0, 1 << 28, (1 << 28) - 1, (1 << 28) + 1, (1 << 29) - 1, 1, 0x5 << 24, 0x11 << 23):
        w = (bits | np.uint64(off)).view(np.float64)
        for sc in (2.0 ** -1, 2.0 ** -20, 2.0 ** -60, 2.0 ** -75, 2.0 ** -120, 2.0 ** -126, 2.0 ** 100):
            parts.append(w * sc)
    # boundaries: binades where the fast paths start and end, and 1 - ulp
    for k in (-149, -127, -126, -125, -75, -74, -73, -22, -21, -20, 127, 128):
        b = np.float64(2.0) ** k
        parts.append(np.array([b, np.nextafter(b, 0), np.nextafter(b, 10), 1.5 * b]))
    parts.append(np.array([0.0, -0.0, 1.0, np.nextafter(1.0, 0.0), 0.5, np.inf, -np.inf, np.nan,
                           np.finfo(np.float64).max, np.finfo(np.float64).tiny, 5e-324,
                           float(np.finfo(np.float32).max), 3.4028235677973366e38]))
    return np.concatenate(parts)


def test_conversions_match_the_fp64_operations(lib):
    x = inputs()
    f, h, l, q, inside = run(lib, x)
    with np.errstate(over="ignore", invalid="ignore"):
        ref_f = x.astype(np.float32)
        ref_l = (x - ref_f.astype(np.float64)).astype(np.float32)
    same = lambda a, b: (a.view(np.uint32) == b.view(np.uint32)) | (np.isnan(a) & np.isnan(b))
    assert same(f, ref_f).all(), x[~same(f, ref_f)][:5]
    assert same(h, ref_f).all(), x[~same(h, ref_f)][:5]
    fin = np.isfinite(x) & np.isfinite(ref_f)
    assert same(l[fin], ref_l[fin]).all(), x[fin][~same(l[fin], ref_l[fin])][:5]
    with np.errstate(invalid="ignore"):
        ref_in = (x >= 0.0) & (x < 1.0)
        with np.errstate(over="ignore"):
            s = x * 2097152.0
        ref_q = np.where(np.isnan(s) | ~(s >= 0.0), 0.0, np.minimum(np.floor(np.where(np.isfinite(s), s, 4e6)),
                                                                      2097151.0)).astype(np.uint32)
    assert (inside == ref_in).all(), x[inside != ref_in][:5]
    assert (q == ref_q).all(), x[q != ref_q][:5]


def test_the_pair_represents_the_double(lib):
    """h + l recovers x to FP32 x FP32 precision (|x - h - l| <= 2^-24 |l|), on positions in [0, 1)."""
    x = np.random.default_rng(3).random(100000)
    _, h, l, _, _ = run(lib, x)
    r = x - h.astype(np.float64) - l.astype(np.float64)
    assert np.all(np.abs(r) <= np.abs(l.astype(np.float64)) * 2.0 ** -24 + 1e-300)


def test_widening_and_order_keys(lib):
    """fmm_f2d equals (double)f for every class of float; the order keys of non-negative doubles sort
    as the values do, with -0.0 keyed as +0.0, and give the value back."""
    rng = np.random.default_rng(5)
    bits = rng.integers(0, 2 ** 32, 200000, dtype=np.uint64).astype(np.uint32)
    special = np.array([0, 0x80000000, 1, 0x807FFFFF, 0x00800000, 0x7F7FFFFF, 0x7F800000, 0xFF800000,
                        0x7FC00000, 0x3F800000], dtype=np.uint32)
    f = np.concatenate([bits, special]).view(np.float32)
    d = np.empty(f.size, np.float64)
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    lib.h_widen(p(f), ctypes.c_longlong(f.size), p(d))
    ref = f.astype(np.float64)
    ok = (d.view(np.uint64) == ref.view(np.uint64)) | (np.isnan(d) & np.isnan(ref))
    assert ok.all(), f[~ok][:5]
    x = np.concatenate([rng.random(50000), rng.random(1000) * 1e-300, [0.0, -0.0, 1.0, 5e-324, np.inf]])
    k = np.empty(x.size, np.uint64)
    back = np.empty(x.size, np.float64)
    lib.h_keys(p(x), ctypes.c_longlong(x.size), p(k), p(back))
    assert (back == x).all()
    o = np.argsort(k, kind="stable")
    assert (np.diff(x[o]) >= 0).all()
    assert k[x.size - 4] == 0 and k[x.size - 5] == 0  # -0.0 and +0.0 share the key of zero
