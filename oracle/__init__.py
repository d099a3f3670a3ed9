"""FP64 CPU oracle for the FMM force solve -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path never calls it, and it
shares no code with the CUDA path (``oracle.c`` is compiled on its own by
``oracle/build.py``).

Python view of the C oracle:

* :func:`direct`      -- softened O(N^2) direct sum (Sec. 2 / Sec. 3.1), the accuracy reference.
* :func:`green_derivs`, :func:`p2m`, :func:`m2p`, :func:`m2l`, :func:`p2l`,
  :func:`l2l`, :func:`l2p` -- the expansion operators of Sec. 3.1 (moments to
  order 4, local expansion to order 5), in multi-index form.
* :func:`direct_periodic`, :func:`ewald_derivs`, :func:`ewald_m2p` -- the
  periodic unit box (Sec. 3.1): the periodic direct sum by Ewald summation, and
  the correction kernel for the copies beyond the replica shell.
* :class:`FMM` -- the plain recursive FMM (tree, moments, checklist walk,
  PP / PC / CC / CP / L2L / L2P), with its tree, lists and local expansions
  exposed for stage-by-stage parity; ``nrep`` makes the box periodic.

``kdk`` holds the rung assignment and kick-drift-kick schedule (Sec. 3.2) and
``mlp`` the FP64 reference of the learned opening criterion's network.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

NMI = 56  # multi-indices with |n| <= 5
NM4 = 35  # multi-indices with |n| <= 4
KINDS = {"pp": 0, "pc": 1, "cc": 2, "cp": 3}

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
        lp = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
        ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
        up = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")
        L.orc_direct.argtypes = [C.c_long, dp, dp, C.c_double, C.c_long, C.c_void_p, dp, dp]
        L.orc_green_derivs.argtypes = [dp, C.c_double, dp]
        L.orc_p2m.argtypes = [C.c_long, dp, dp, dp, dp]
        L.orc_m2p.argtypes = [dp, dp, dp, C.c_double, dp, dp]
        L.orc_m2l.argtypes = [dp, dp, dp, C.c_double, dp]
        L.orc_p2l.argtypes = [C.c_double, dp, dp, C.c_double, dp]
        L.orc_l2l.argtypes = [dp, dp, dp]
        L.orc_l2p.argtypes = [dp, dp, dp, dp]
        L.orc_multi_index.argtypes = [ip]
        L.orc_ewald_derivs.argtypes = [dp, C.c_int, C.c_double, dp]
        L.orc_ewald_m2p.argtypes = [dp, dp, dp, C.c_int, C.c_double, dp, dp]
        L.orc_direct_periodic.argtypes = [C.c_long, dp, dp, C.c_double, C.c_int, C.c_double, C.c_long,
                                          C.c_void_p, dp, dp]
        L.orc_fmm_create.restype = C.c_void_p
        L.orc_fmm_create.argtypes = [C.c_long, dp, dp, C.c_void_p, C.c_double, C.c_double, C.c_int, C.c_int]
        L.orc_fmm_create_periodic.restype = C.c_void_p
        L.orc_fmm_create_periodic.argtypes = [C.c_long, dp, dp, C.c_void_p, C.c_double, C.c_double, C.c_int,
                                              C.c_int, C.c_int]
        L.orc_fmm_entry_shifts.argtypes = [C.c_void_p, C.c_int, ip]
        L.orc_fmm_eval.argtypes = [C.c_void_p, C.c_int, dp, dp]
        L.orc_fmm_ncell.restype = C.c_long
        L.orc_fmm_ncell.argtypes = [C.c_void_p]
        L.orc_fmm_ngroup.restype = C.c_long
        L.orc_fmm_ngroup.argtypes = [C.c_void_p]
        L.orc_fmm_nentries.restype = C.c_long
        L.orc_fmm_nentries.argtypes = [C.c_void_p, C.c_int]
        L.orc_fmm_perm.argtypes = [C.c_void_p, lp]
        L.orc_fmm_keys.argtypes = [C.c_void_p, up]
        L.orc_fmm_cells.argtypes = [C.c_void_p, lp, lp, lp, lp, lp, dp, dp, dp, dp, dp, dp]
        L.orc_fmm_entries.argtypes = [C.c_void_p, C.c_int, lp, lp, lp]
        L.orc_fmm_groups.argtypes = [C.c_void_p, lp, dp]
        L.orc_fmm_counts.argtypes = [C.c_void_p, lp]
        L.orc_fmm_free.argtypes = [C.c_void_p]
        L.orc_num_threads.restype = C.c_int
        _lib = L
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads() -> int:
    return int(lib().orc_num_threads())


def multi_index() -> np.ndarray:
    out = np.zeros(3 * NMI, dtype=np.int32)
    lib().orc_multi_index(out)
    return out.reshape(NMI, 3)


def direct(pos, mass, eps, sinks=None):
    """FP64 direct sum.  pos (3, N), mass (N,).  Returns acc (3, S), pot (S,) for the sinks."""
    pos = _f64(pos)
    mass = _f64(mass)
    n = pos.shape[1]
    if sinks is None:
        ns, sp = n, None
        keep = None
    else:
        keep = np.ascontiguousarray(sinks, dtype=np.int64)
        ns, sp = keep.shape[0], keep.ctypes.data
    acc = np.zeros(3 * ns)
    pot = np.zeros(ns)
    lib().orc_direct(n, pos.reshape(-1), mass, float(eps), ns, sp, acc, pot)
    return acc.reshape(3, ns), pot


def direct_periodic(pos, mass, eps, sinks=None, nrep=1, alpha=8.0):
    """FP64 periodic direct sum in the unit box: the softened kernel on the copies inside the
    replica shell |n|_inf <= nrep, the Newtonian Ewald sum beyond (Ewald parameter alpha; the
    result does not depend on it).  Returns acc (3, S), pot (S,) for the sinks."""
    pos = _f64(pos)
    mass = _f64(mass)
    n = pos.shape[1]
    if sinks is None:
        ns, sp, keep = n, None, None
    else:
        keep = np.ascontiguousarray(sinks, dtype=np.int64)
        ns, sp = keep.shape[0], keep.ctypes.data
    acc = np.zeros(3 * ns)
    pot = np.zeros(ns)
    lib().orc_direct_periodic(n, pos.reshape(-1), mass, float(eps), int(nrep), float(alpha), ns, sp, acc, pot)
    return acc.reshape(3, ns), pot


def ewald_derivs(r, nrep=1, alpha=3.0):
    """D^n F(r), |n| <= 5: F is the periodic potential of a unit mass (background subtracted)
    less the Newtonian copies inside the replica shell.  Offsets with |r_a| < 1."""
    D = np.zeros(NMI)
    lib().orc_ewald_derivs(_f64(r), int(nrep), float(alpha), D)
    return D


def ewald_m2p(M, z, x, nrep=1, alpha=3.0):
    """The correction for the copies beyond the replica shell at x, from moments M about z."""
    acc = np.zeros(3)
    pot = np.zeros(1)
    lib().orc_ewald_m2p(_f64(M), _f64(z), _f64(x), int(nrep), float(alpha), acc, pot)
    return acc, pot[0]


def green_derivs(r, eps2):
    D = np.zeros(NMI)
    lib().orc_green_derivs(_f64(r), float(eps2), D)
    return D


def p2m(pos, mass, c):
    pos = _f64(pos)
    M = np.zeros(NM4)
    lib().orc_p2m(pos.shape[1], pos.reshape(-1), _f64(mass), _f64(c), M)
    return M


def m2p(M, z, x, eps2):
    acc = np.zeros(3)
    pot = np.zeros(1)
    lib().orc_m2p(_f64(M), _f64(z), _f64(x), float(eps2), acc, pot)
    return acc, pot[0]


def m2l(M, z, c, eps2):
    L = np.zeros(NMI)
    lib().orc_m2l(_f64(M), _f64(z), _f64(c), float(eps2), L)
    return L


def p2l(m, x, c, eps2):
    L = np.zeros(NMI)
    lib().orc_p2l(float(m), _f64(x), _f64(c), float(eps2), L)
    return L


def l2l(L, t):
    out = np.zeros(NMI)
    lib().orc_l2l(_f64(L), _f64(t), out)
    return out


def l2p(L, u):
    acc = np.zeros(3)
    pot = np.zeros(1)
    lib().orc_l2p(_f64(L), _f64(u), acc, pot)
    return acc, pot[0]


class FMM:
    """Plain recursive FMM on the CPU (FP64 arithmetic, single-precision decisions).

    ``nrep`` makes the unit box periodic: the walk starts from the root and its copies
    |n|_inf <= nrep (26 for 1, 124 for 2), and ``forces`` adds the Ewald correction for the
    copies beyond (term bit 8)."""

    def __init__(self, pos, mass, eps, theta, bucket=16, group=64, active=None, nrep=None):
        pos = _f64(pos)
        self.n = pos.shape[1]
        self._act = None
        ap = None
        if active is not None:
            self._act = np.ascontiguousarray(active, dtype=np.uint8)
            ap = self._act.ctypes.data
        if nrep is None:
            self.h = lib().orc_fmm_create(self.n, pos.reshape(-1), _f64(mass), ap, float(eps), float(theta),
                                          int(bucket), int(group))
        else:
            self.h = lib().orc_fmm_create_periodic(self.n, pos.reshape(-1), _f64(mass), ap, float(eps),
                                                   float(theta), int(bucket), int(group), int(nrep))
            if not self.h:
                raise ValueError("nrep must be 0, 1 or 2")
        self.eps, self.theta, self.bucket, self.group, self.nrep = eps, theta, bucket, group, nrep

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            lib().orc_fmm_free(h)
            self.h = None

    def forces(self, terms=None, fill=0.0):
        if terms is None:
            terms = 7 if self.nrep is None else 15
        acc = np.full(3 * self.n, fill)
        pot = np.full(self.n, fill)
        lib().orc_fmm_eval(self.h, int(terms), acc, pot)
        return acc.reshape(3, self.n), pot

    def perm(self):
        p = np.zeros(self.n, dtype=np.int64)
        lib().orc_fmm_perm(self.h, p)
        return p

    def keys(self):
        k = np.zeros(self.n, dtype=np.uint64)
        lib().orc_fmm_keys(self.h, k)
        return k

    def cells(self):
        nc = lib().orc_fmm_ncell(self.h)
        d = dict(first=np.zeros(nc, np.int64), count=np.zeros(nc, np.int64), parent=np.zeros(nc, np.int64),
                 child=np.zeros(2 * nc, np.int64), nact=np.zeros(nc, np.int64), mass=np.zeros(nc),
                 com=np.zeros(3 * nc), lo=np.zeros(3 * nc), hi=np.zeros(3 * nc), bmax=np.zeros(nc),
                 mom=np.zeros(NM4 * nc))
        lib().orc_fmm_cells(self.h, d["first"], d["count"], d["parent"], d["child"], d["nact"], d["mass"],
                            d["com"], d["lo"], d["hi"], d["bmax"], d["mom"])
        d["child"] = d["child"].reshape(nc, 2)
        for k in ("com", "lo", "hi"):
            d[k] = d[k].reshape(nc, 3)
        d["mom"] = d["mom"].reshape(nc, NM4)
        return d

    def entries(self, kind):
        k = KINDS[kind]
        n = lib().orc_fmm_nentries(self.h, k)
        s, f, c = (np.zeros(n, np.int64) for _ in range(3))
        lib().orc_fmm_entries(self.h, k, s, f, c)
        return s, f, c

    def shifts(self, kind):
        """The periodic copy of each entry's source (rows (sx, sy, sz)), in the order of entries()."""
        k = KINDS[kind]
        n = lib().orc_fmm_nentries(self.h, k)
        out = np.zeros(3 * n, np.int32)
        lib().orc_fmm_entry_shifts(self.h, k, out)
        return out.reshape(n, 3)

    def groups(self):
        n = lib().orc_fmm_ngroup(self.h)
        cell = np.zeros(n, np.int64)
        L = np.zeros(NMI * n)
        lib().orc_fmm_groups(self.h, cell, L)
        return cell, L.reshape(n, NMI)

    def counts(self):
        out = np.zeros(8, np.int64)
        lib().orc_fmm_counts(self.h, out)
        keys = ["pp_pairs", "pc_pairs", "cc", "cp", "groups", "cells", "buckets", "depth"]
        return dict(zip(keys, (int(v) for v in out)))
