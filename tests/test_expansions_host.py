"""The CUDA path's generated expansion operators (csrc/expansions.cuh), compiled for the host
with g++ and checked against the oracle's independent FP64 operators.

Covered: moment building (P2M, M2M and traces), the particle-cell body in its scalar and FP32x2
forms, and the local expansions (M2L, P2L, L2L, each followed by L2P). The header is the one the kernels include. On the host:
- the FP32x2 intrinsics are per-component fmaf / add / multiply, which is how the CUDA
  documentation defines them;
- the reciprocal square root is 1/sqrtf.

Both sides evaluate the same Plummer-softened Taylor expansion, the GPU's in FP32 through
scaled derivatives and trace contractions, the oracle's in FP64 through multi-index sums. So
they agree to FP32 rounding, measured at <= 3e-7 here, so rtol 3e-6. Six of the sinks sit at
2.5 b_max in different directions. There, a 1% error in 28 of the record's 31 moment components
shifts some sink's force by more than that; the other three are too small in this cluster to
matter.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1609_08621_gb300", "csrc")

HARNESS = r"""
#include <cmath>
#define __device__
#define __forceinline__ inline
#define __restrict__ __restrict
struct float2 { float x, y; };
static inline float2 make_float2(float a, float b) { float2 r; r.x = a; r.y = b; return r; }
static inline float2 __ffma2_rn(float2 a, float2 b, float2 c) { return make_float2(fmaf(a.x, b.x, c.x), fmaf(a.y, b.y, c.y)); }
static inline float2 __fadd2_rn(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
static inline float2 __fmul2_rn(float2 a, float2 b) { return make_float2(a.x * b.x, a.y * b.y); }
#include "expansions.cuh"
extern "C" {
void h_record(int k, const float* y, const float* m, float* R) {
    for (int i = 0; i < FMM_NREC; i++) R[i] = 0.0f;
    for (int j = 0; j < k; j++) fmm_p2m_acc(m[j], y[3 * j], y[3 * j + 1], y[3 * j + 2], R);
    fmm_moment_traces(R);
}
void h_pc(const float* R, float rx, float ry, float rz, float eps2, float* out) {
    float ax = 0.0f, ay = 0.0f, az = 0.0f, phi = 0.0f;
    fmm_pc_acc(R, rx, ry, rz, eps2, ax, ay, az, phi);
    out[0] = ax; out[1] = ay; out[2] = az; out[3] = phi;
}
void h_pc2(const float* R, const float* r0, const float* r1, float eps2, float* out) {
    float2 ax = make_float2(0.0f, 0.0f), ay = ax, az = ax, pp = ax;
    fmm_pc_acc2(R, make_float2(r0[0], r1[0]), make_float2(r0[1], r1[1]), make_float2(r0[2], r1[2]),
                make_float2(eps2, eps2), ax, ay, az, pp);
    out[0] = ax.x; out[1] = ay.x; out[2] = az.x; out[3] = -pp.x;
    out[4] = ax.y; out[5] = ay.y; out[6] = az.y; out[7] = -pp.y;
}
void h_m2m(const float* Rc, float tx, float ty, float tz, float* Mp) {
    fmm_m2m_acc(Rc, tx, ty, tz, Mp);
}
void h_traces(float* R) { fmm_moment_traces(R); }
void h_p2l_l2p(float m, float rx, float ry, float rz, float eps2, float ux, float uy, float uz, float* out) {
    float L[FMM_NL];
    for (int i = 0; i < FMM_NL; i++) L[i] = 0.0f;
    fmm_p2l_acc(m, rx, ry, rz, eps2, L);
    float ax = 0.0f, ay = 0.0f, az = 0.0f, phi = 0.0f;
    fmm_l2p_acc(L, ux, uy, uz, ax, ay, az, phi);
    out[0] = ax; out[1] = ay; out[2] = az; out[3] = phi;
}
void h_m2l_l2l_l2p(const float* R, float rx, float ry, float rz, float eps2, float tx, float ty, float tz, float ux,
                   float uy, float uz, float* out) {
    float L[FMM_NL], Lo[FMM_NL];
    for (int i = 0; i < FMM_NL; i++) L[i] = 0.0f;
    fmm_m2l_acc(R, rx, ry, rz, eps2, L);
    fmm_l2l(L, tx, ty, tz, Lo);
    float ax = 0.0f, ay = 0.0f, az = 0.0f, phi = 0.0f;
    fmm_l2p_acc(Lo, ux, uy, uz, ax, ay, az, phi);
    out[0] = ax; out[1] = ay; out[2] = az; out[3] = phi;
}
void h_m2l_l2p(const float* R, float rx, float ry, float rz, float eps2, float ux, float uy, float uz, float* out) {
    float L[FMM_NL];
    for (int i = 0; i < FMM_NL; i++) L[i] = 0.0f;
    fmm_m2l_acc(R, rx, ry, rz, eps2, L);
    float ax = 0.0f, ay = 0.0f, az = 0.0f, phi = 0.0f;
    fmm_l2p_acc(L, ux, uy, uz, ax, ay, az, phi);
    out[0] = ax; out[1] = ay; out[2] = az; out[3] = phi;
}
}
"""

F = ctypes.POINTER(ctypes.c_float)


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("expansions_host")
    src = d / "harness.cpp"
    src.write_text(HARNESS)
    so = d / "libharness.so"
    subprocess.run([cxx, "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-I", CSRC, str(src), "-o", str(so)],
                   check=True, capture_output=True)
    return ctypes.CDLL(str(so))


def _f(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    return a, a.ctypes.data_as(F)


def _cluster(seed, k=30, b=0.01):
    """k particles within b of their FP64 centre of mass z; the record's offsets are fl(x - z)."""
    rng = np.random.default_rng(seed)
    pos = 0.5 + b * (rng.random((3, k)) - 0.5)
    m = (0.5 + rng.random(k)) / k
    z = (pos * m).sum(axis=1) / m.sum()
    return pos, m, z


def _record(lib, pos, m, z):
    y, yp = _f((pos - z[:, None]).T.reshape(-1))
    mm, mp = _f(m)
    R, Rp = _f(np.zeros(44))
    lib.h_record(ctypes.c_int(m.size), yp, mp, Rp)
    return R, Rp


@pytest.mark.parametrize("eps", [0.0, 2e-3])
def test_particle_cell_body_matches_the_oracle(lib, eps):
    pos, m, z = _cluster(1)
    R, Rp = _record(lib, pos, m, z)
    M = oracle.p2m(pos, m, z)
    rng = np.random.default_rng(2)
    for d in (0.02,) * 6 + (0.05, 0.1, 0.3):
        dirn = rng.normal(size=3)
        x = z + d * dirn / np.linalg.norm(dirn)
        out, op = _f(np.zeros(4))
        r = (x - z).astype(np.float32)
        lib.h_pc(Rp, ctypes.c_float(r[0]), ctypes.c_float(r[1]), ctypes.c_float(r[2]), ctypes.c_float(eps * eps), op)
        # the sink offset is rounded to FP32 on the GPU side: compare at that position
        ref, rp = oracle.m2p(M, z, z + r.astype(np.float64), eps * eps)
        assert np.allclose(out[:3], ref, rtol=3e-6, atol=3e-6 * np.linalg.norm(ref)), (d, out[:3], ref)
        assert out[3] == pytest.approx(rp, rel=3e-6)


def test_paired_body_matches_the_scalar_body(lib):
    """fmm_pc_acc2 evaluates two sinks with the same arithmetic as fmm_pc_acc; only the fused
    multiply-adds are grouped differently, so they agree to FP32 rounding."""
    pos, m, z = _cluster(3)
    R, Rp = _record(lib, pos, m, z)
    rng = np.random.default_rng(4)
    for _ in range(20):
        r0 = (rng.normal(size=3) * 0.08).astype(np.float32)
        r1 = (rng.normal(size=3) * 0.2).astype(np.float32)
        o2, o2p = _f(np.zeros(8))
        lib.h_pc2(Rp, _f(r0)[1], _f(r1)[1], ctypes.c_float(1e-6), o2p)
        for h, r in ((0, r0), (1, r1)):
            o1, o1p = _f(np.zeros(4))
            lib.h_pc(Rp, ctypes.c_float(r[0]), ctypes.c_float(r[1]), ctypes.c_float(r[2]), ctypes.c_float(1e-6), o1p)
            a2, a1 = o2[4 * h: 4 * h + 3], o1[:3]
            assert np.allclose(a2, a1, rtol=3e-6, atol=3e-6 * np.linalg.norm(a1))
            assert o2[4 * h + 3] == pytest.approx(o1[3], rel=3e-6)


def test_m2l_then_l2p_matches_the_oracle(lib):
    pos, m, z = _cluster(5)
    R, Rp = _record(lib, pos, m, z)
    M = oracle.p2m(pos, m, z)
    c = z + np.array([0.13, -0.08, 0.06])
    eps2 = 1e-6
    rng = np.random.default_rng(6)
    rc = (c - z).astype(np.float32)
    c = z + rc.astype(np.float64)  # the centre offset the GPU side sees
    L = oracle.m2l(M, z, c, eps2)
    for _ in range(5):
        u = (rng.normal(size=3) * 0.01).astype(np.float32)
        out, op = _f(np.zeros(4))
        lib.h_m2l_l2p(Rp, ctypes.c_float(rc[0]), ctypes.c_float(rc[1]), ctypes.c_float(rc[2]), ctypes.c_float(eps2),
                      ctypes.c_float(u[0]), ctypes.c_float(u[1]), ctypes.c_float(u[2]), op)
        ref, rp = oracle.l2p(L, u.astype(np.float64))
        assert np.allclose(out[:3], ref, rtol=3e-6, atol=3e-6 * np.linalg.norm(ref)), (out[:3], ref)
        assert out[3] == pytest.approx(rp, rel=3e-6)


def _c(v):
    return [ctypes.c_float(float(x)) for x in v]


def test_m2m_shift_matches_the_parent_moments(lib):
    """Two sub-clusters, each with moments about its own centre, shifted to the parent's centre:
    the parent record gives the field of the oracle's moments of all particles about that centre."""
    pos, m, zp = _cluster(7, k=40, b=0.012)
    halves = (pos[0] < zp[0], pos[0] >= zp[0])
    Mp, Mpp = _f(np.zeros(44))
    for h in halves:
        ph, mh = pos[:, h], m[h]
        zc = (ph * mh).sum(axis=1) / mh.sum()
        Rc, Rcp = _record(lib, ph, mh, zc)
        lib.h_m2m(Rcp, *_c((zc - zp).astype(np.float32)), Mpp)
    lib.h_traces(Mpp)
    M = oracle.p2m(pos, m, zp)
    rng = np.random.default_rng(8)
    for d in (0.03, 0.1):
        dirn = rng.normal(size=3)
        r = (d * dirn / np.linalg.norm(dirn)).astype(np.float32)
        out, op = _f(np.zeros(4))
        lib.h_pc(Mpp, *_c(r), ctypes.c_float(1e-6), op)
        ref, rp = oracle.m2p(M, zp, zp + r.astype(np.float64), 1e-6)
        assert np.allclose(out[:3], ref, rtol=3e-6, atol=3e-6 * np.linalg.norm(ref)), (out[:3], ref)
        assert out[3] == pytest.approx(rp, rel=3e-6)


def test_p2l_then_l2p_matches_the_oracle(lib):
    rng = np.random.default_rng(9)
    c = np.array([0.5, 0.5, 0.5])
    for _ in range(4):
        x = c + rng.normal(size=3) * 0.1
        m = float(rng.random() + 0.1)
        r = (c - x).astype(np.float32)
        u = (rng.normal(size=3) * 0.01).astype(np.float32)
        out, op = _f(np.zeros(4))
        lib.h_p2l_l2p(ctypes.c_float(m), *_c(r), ctypes.c_float(1e-6), *_c(u), op)
        L = oracle.p2l(np.float32(m), c - r.astype(np.float64), c, 1e-6)
        ref, rp = oracle.l2p(L, u.astype(np.float64))
        assert np.allclose(out[:3], ref, rtol=3e-6, atol=3e-6 * np.linalg.norm(ref)), (out[:3], ref)
        assert out[3] == pytest.approx(rp, rel=3e-6)


def test_l2l_shift_then_l2p_matches_the_oracle(lib):
    """A local expansion shifted to a child's centre (the groups' ancestor sums): exact for a
    polynomial of degree 5, so it equals the oracle's expansion evaluated at t + u."""
    pos, m, z = _cluster(10)
    R, Rp = _record(lib, pos, m, z)
    M = oracle.p2m(pos, m, z)
    rc = np.array([0.15, 0.1, -0.07], np.float32)
    c = z + rc.astype(np.float64)
    L = oracle.m2l(M, z, c, 1e-6)
    rng = np.random.default_rng(11)
    for _ in range(4):
        t = (rng.normal(size=3) * 0.01).astype(np.float32)
        u = (rng.normal(size=3) * 0.004).astype(np.float32)
        out, op = _f(np.zeros(4))
        lib.h_m2l_l2l_l2p(Rp, *_c(rc), ctypes.c_float(1e-6), *_c(t), *_c(u), op)
        ref, rp = oracle.l2p(L, t.astype(np.float64) + u.astype(np.float64))
        assert np.allclose(out[:3], ref, rtol=3e-6, atol=3e-6 * np.linalg.norm(ref)), (out[:3], ref)
        assert out[3] == pytest.approx(rp, rel=3e-6)
