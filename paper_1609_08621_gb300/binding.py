"""ctypes binding of the C ABI in ``include/fmm.h`` (argument marshalling only).

Every computation happens in the CUDA library ``_build/libfmm_gb300.so``; if it is
missing and cannot be built, loading raises -- there is no CPU fallback.  PyTorch is
used only for device memory and streams: tensors are passed by their data pointers
after their dtype, device, shape and contiguity are checked.

The functions keep the C names (``fmm_create``, ``fmm_compute_forces``, ...);
:class:`Context` is a small owner of one ``fmm_ctx``.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

FMM_OK = 0
STATUS = {0: "FMM_OK", -1: "FMM_ERR_ARG", -2: "FMM_ERR_OOM", -3: "FMM_ERR_CUDA", -4: "FMM_ERR_TIMEOUT",
          -5: "FMM_ERR_STATE", -6: "FMM_ERR_NUMERIC"}
FMM_OK, FMM_ERR_ARG, FMM_ERR_OOM, FMM_ERR_CUDA, FMM_ERR_TIMEOUT, FMM_ERR_STATE, FMM_ERR_NUMERIC = 0, -1, -2, -3, -4, -5, -6
KIND = {"pp": 0, "pc": 1, "cc": 2, "cp": 3}


class FmmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class fmm_params(C.Structure):
    _fields_ = [("theta", C.c_double), ("eps", C.c_double), ("bucket", C.c_int), ("group", C.c_int),
                ("criterion", C.c_int), ("accumulate", C.c_int), ("terms", C.c_int), ("list_chunk", C.c_int),
                ("spin_limit", C.c_longlong), ("mlp_tau", C.c_double), ("band_lo", C.c_double),
                ("band_hi", C.c_double), ("nrep", C.c_int), ("mlp_margin", C.c_double)]


class fmm_stats(C.Structure):
    _fields_ = [(k, C.c_longlong) for k in ("n", "n_active", "n_cells", "n_buckets", "n_groups", "n_levels",
                                             "n_pp_pairs", "n_pc_pairs", "n_cc", "n_cp", "n_pp_entries",
                                             "n_pc_entries")] + \
               [(k, C.c_double) for k in ("ms_tree", "ms_walk", "ms_pp", "ms_pc", "ms_l2p", "ms_total",
                                          "paper_flops", "kernel_flops_pp", "kernel_flops_pc")] + \
               [("retries", C.c_int), ("n_launches", C.c_int), ("n_learned", C.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load the CUDA library (building it with nvcc if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing:
        path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing; run __graft_entry__.build()")
    L = C.CDLL(path)
    vp, ll, d, i = C.c_void_p, C.c_longlong, C.c_double, C.c_int
    sig = {
        "fmm_default_params": (i, [C.POINTER(fmm_params)]),
        "fmm_create": (i, [C.POINTER(vp), i, vp]),
        "fmm_destroy": (None, [vp]),
        "fmm_set_params": (i, [vp, C.POINTER(fmm_params)]),
        "fmm_get_params": (i, [vp, C.POINTER(fmm_params)]),
        "fmm_build_tree": (i, [vp, vp, vp, vp, ll, C.POINTER(fmm_params)]),
        "fmm_compute_forces": (i, [vp, vp, vp, vp, ll, d, d, vp, vp]),
        "fmm_compute_forces_host": (i, [vp, vp, vp, vp, ll, d, d, vp, vp]),
        "fmm_compute_forces_batch": (i, [vp, vp, vp, vp, ll, vp, i, d, d, vp, vp]),
        "fmm_kick_drift": (i, [vp, vp, vp, vp, vp, vp, ll, d, d, i, i, i]),
        "fmm_assign_rungs": (i, [vp, vp, vp, ll, d, d, i]),
        "fmm_set_fixed_sources": (i, [vp, vp, vp, vp, vp, ll, i, d]),
        "fmm_compute_forces_dual": (i, [vp, vp, vp, vp, ll, d, d, vp, vp]),
        "fmm_get_stats": (i, [vp, C.POINTER(fmm_stats)]),
        "fmm_last_error": (C.c_char_p, []),
        "fmm_flops_per_pc": (d, []),
        "fmm_tree_info": (i, [vp, C.POINTER(ll), C.POINTER(ll), C.POINTER(ll), C.POINTER(ll), C.POINTER(ll)]),
        "fmm_export_order": (i, [vp, vp, vp]),
        "fmm_export_cells": (i, [vp] + [vp] * 11),
        "fmm_export_lists": (i, [vp, i, C.POINTER(ll), vp, vp, vp, ll]),
        "fmm_export_list_shifts": (i, [vp, i, C.POINTER(ll), vp, ll]),
        "fmm_export_locals": (i, [vp, vp, vp, ll]),
        "fmm_multi_index": (i, [vp, vp]),
        "fmm_export_walk_levels": (i, [vp, vp, i, C.POINTER(i)]),
        "fmm_mlp_load": (i, [vp, vp, ll]),
        "fmm_mlp_get": (i, [vp, vp, ll]),
        "fmm_mlp_predict": (i, [vp, vp, ll, vp]),
        "fmm_mlp_gradient": (i, [vp, vp, vp, ll, vp, vp]),
        "fmm_mlp_train": (i, [vp, vp, vp, ll, i, i, C.c_float, C.c_uint, vp]),
        "fmm_mlp_audit": (i, [vp, vp, vp, ll, d, d, d, d, vp, ll, vp, vp, C.POINTER(ll)]),
        "fmm_mlp_audit_pairs": (i, [vp, vp, vp, vp, vp, ll]),
        "fmm_morton_order_static": (i, [vp, ll, vp, vp, vp]),
        "fmm_debug_fail_allocations": (i, [ll]),
        "fmm_compute_forces_i32": (i, [vp, vp, vp, vp, ll, d, d, vp, vp]),
        "fmm_kick_drift_i32": (i, [vp, vp, vp, vp, vp, vp, ll, d, d, i, i, i]),
        "fmm_memory_info": (i, [vp, C.POINTER(ll), C.POINTER(ll)]),
        "fmm_debug_walk_capacity": (i, [vp, ll, ll]),
        "fmm_debug_local_side": (i, [vp, ll]),
        "fmm_set_graphs": (i, [vp, i]),
        "fmm_graph_info": (i, [vp, C.POINTER(i), C.POINTER(ll)]),
        "fmm_autotune": (i, [vp, vp, vp, ll, vp, i, d, d, vp, i, i, vp, C.POINTER(fmm_params), C.POINTER(C.c_float)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(st):
    if st != FMM_OK:
        raise FmmError(st, load().fmm_last_error().decode())


def _ptr(t, dtype, n=None, name="tensor", allow_none=False):
    """Data pointer of a contiguous CUDA tensor of the given torch dtype."""
    if t is None:
        if allow_none:
            return None
        raise ValueError(f"{name} must not be None")
    import torch

    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if n is not None and t.numel() != n:
        raise ValueError(f"{name} must have {n} elements, got {t.numel()}")
    return t.data_ptr()


def _hptr(a, dtype, n=None, name="array", allow_none=False):
    if a is None:
        if allow_none:
            return None
        raise ValueError(f"{name} must not be None")
    if not isinstance(a, np.ndarray) or a.dtype != dtype or not a.flags["C_CONTIGUOUS"]:
        raise TypeError(f"{name} must be a C-contiguous numpy array of {dtype}")
    if n is not None and a.size != n:
        raise ValueError(f"{name} must have {n} elements, got {a.size}")
    return a.ctypes.data


def fmm_default_params() -> fmm_params:
    p = fmm_params()
    _check(load().fmm_default_params(C.byref(p)))
    return p


def fmm_flops_per_pc() -> float:
    return float(load().fmm_flops_per_pc())


def fmm_multi_index():
    loc = np.zeros(56 * 3, np.int32)
    mom = np.zeros(32 * 3, np.int32)
    _check(load().fmm_multi_index(loc.ctypes.data, mom.ctypes.data))
    return loc.reshape(56, 3), mom.reshape(32, 3)


STATIC_ORDER_MAX_N = 1048576


def morton_order_static(pos, keys, order, stream=None):
    """Allocation-free Morton order (fmm_morton_order_static): pos is a (3, n) or 3n float64
    CUDA tensor; the sorted keys (int64 holding the uint64 keys) and the order (int32 holding
    the uint32 indices) are written into the caller's n-element CUDA tensors.  Nothing is
    allocated on this path; the call returns once the stream has finished."""
    import torch

    n = keys.numel()
    devs = {t.device for t in (pos, keys, order)}
    if len(devs) != 1:
        raise ValueError(f"pos, keys and order must be on one device, got {sorted(str(d) for d in devs)}")
    # the C call runs on the current device: make it the tensors' device for the call
    with torch.cuda.device(keys.device):
        if stream is None:
            stream = torch.cuda.current_stream(keys.device)
        _check(load().fmm_morton_order_static(_ptr(pos, torch.float64, 3 * n, "pos"), n,
                                              _ptr(keys, torch.int64, n, "keys"),
                                              _ptr(order, torch.int32, n, "order"), C.c_void_p(stream.cuda_stream)))


def debug_fail_allocations(after):
    """fmm_debug_fail_allocations: the calling thread's device allocations after the next `after`
    fail as out of memory (after < 0: off).  A test hook for the recovery path."""
    _check(load().fmm_debug_fail_allocations(int(after)))


class Context:
    """One fmm_ctx on a CUDA device, bound to a CUDA stream (torch's current stream by default)."""

    def __init__(self, device: int = 0, stream=None, **params):
        import torch

        self.device = int(device)
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        self.stream = stream
        h = C.c_void_p()
        _check(load().fmm_create(C.byref(h), self.device, C.c_void_p(stream.cuda_stream)))
        self.h = h
        if params:
            self.set_params(**params)

    def close(self):
        """fmm_destroy: release everything the context owns (idempotent)."""
        if getattr(self, "h", None):
            load().fmm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- parameters
    def get_params(self) -> fmm_params:
        """fmm_get_params: the context's current parameters."""
        p = fmm_params()
        _check(load().fmm_get_params(self.h, C.byref(p)))
        return p

    def set_params(self, **kw):
        """fmm_set_params with the given fields changed (bucket, group, list_chunk, criterion,
        accumulate, mlp_tau, ...); the others keep their values."""
        p = self.get_params()
        for k, v in kw.items():
            setattr(p, k, v)
        _check(load().fmm_set_params(self.h, C.byref(p)))

    # -- solve
    def build_tree(self, pos, mass, active=None, params=None):
        """fmm_build_tree: keys, sort, tree and upward pass only.  pos (3N float64 SoA), mass (N
        float32), active (N uint8 or None) -- CUDA tensors."""
        import torch

        n = mass.numel()
        pp = C.byref(params) if params is not None else None
        _check(load().fmm_build_tree(self.h, _ptr(pos, torch.float64, 3 * n, "pos"),
                                     _ptr(mass, torch.float32, n, "mass"),
                                     _ptr(active, torch.uint8, n, "active", True), n, pp))

    def compute_forces(self, pos, mass, eps, theta, acc, pot=None, active=None):
        """pos (3N float64 SoA), mass (N float32), acc out (3N float32), pot out (N float32) -- CUDA tensors."""
        import torch

        n = mass.numel()
        _check(load().fmm_compute_forces(self.h, _ptr(pos, torch.float64, 3 * n, "pos"),
                                         _ptr(mass, torch.float32, n, "mass"),
                                         _ptr(active, torch.uint8, n, "active", True), n, float(eps), float(theta),
                                         _ptr(acc, torch.float32, 3 * n, "acc"),
                                         _ptr(pot, torch.float32, n, "pot", True)))

    def compute_forces_batch(self, pos, mass, box_offsets, eps, theta, acc, pot=None, active=None):
        """Several isolated boxes in one solve; box_offsets: int64 numpy array of nbox + 1 offsets."""
        import torch

        n = mass.numel()
        off = np.ascontiguousarray(box_offsets, dtype=np.int64)
        _check(load().fmm_compute_forces_batch(self.h, _ptr(pos, torch.float64, 3 * n, "pos"),
                                               _ptr(mass, torch.float32, n, "mass"),
                                               _ptr(active, torch.uint8, n, "active", True), n, off.ctypes.data,
                                               off.size - 1, float(eps), float(theta),
                                               _ptr(acc, torch.float32, 3 * n, "acc"),
                                               _ptr(pot, torch.float32, n, "pot", True)))

    def set_graphs(self, enable=True):
        """fmm_set_graphs: replay the whole solve as a CUDA graph while its arguments and buffers
        stay the same (captured after an eager solve)."""
        _check(load().fmm_set_graphs(self.h, 1 if enable else 0))

    def graph_info(self):
        """fmm_graph_info: whether a graph is captured, and how many solves replayed it."""
        cap, rep = C.c_int(), C.c_longlong()
        _check(load().fmm_graph_info(self.h, C.byref(cap), C.byref(rep)))
        return {"captured": bool(cap.value), "replays": rep.value}

    def autotune(self, pos, mass, eps, theta, acc, candidates=None, reps=2, box_offsets=None):
        """Time each candidate (list of (bucket, group, list_chunk)) or the built-in grid; the
        fastest stays in the context.  Returns (best fmm_params, ms per solve)."""
        import torch

        n = mass.numel()
        arr, nc = None, 0
        if candidates is not None:
            arr = (fmm_params * len(candidates))()
            for k, (b, g, ch) in enumerate(candidates):
                arr[k].bucket, arr[k].group, arr[k].list_chunk = b, g, ch
            nc = len(candidates)
        off, nbox = None, 1
        if box_offsets is not None:
            off = np.ascontiguousarray(box_offsets, dtype=np.int64)
            nbox = off.size - 1
        best = fmm_params()
        ms = C.c_float()
        _check(load().fmm_autotune(self.h, _ptr(pos, torch.float64, 3 * n, "pos"), _ptr(mass, torch.float32, n, "mass"),
                                   n, None if off is None else off.ctypes.data, nbox, float(eps), float(theta),
                                   None if arr is None else C.cast(arr, C.c_void_p), nc, int(reps),
                                   _ptr(acc, torch.float32, 3 * n, "acc"), C.byref(best), C.byref(ms)))
        return best, float(ms.value)

    def compute_forces_host(self, pos, mass, eps, theta, acc, pot=None, active=None):
        """Host (numpy) buffers; copies happen inside the library call."""
        n = mass.size
        _check(load().fmm_compute_forces_host(self.h, _hptr(pos, np.float64, 3 * n, "pos"),
                                              _hptr(mass, np.float32, n, "mass"),
                                              _hptr(active, np.uint8, n, "active", True), n, float(eps),
                                              float(theta), _hptr(acc, np.float32, 3 * n, "acc"),
                                              _hptr(pot, np.float32, n, "pot", True)))

    def kick_drift(self, pos, vel, acc, rung, active_next, eps, dt0, max_rung, substep, closing):
        """fmm_kick_drift: one substep of the hierarchical KDK (Sec. 3.2) -- closing half kick (when
        closing), rung reassignment and opening half kick of the particles active at substep, then
        the drift of all; active_next marks the particles whose forces come next.  pos, vel (3N
        float64), acc (3N float32), rung and active_next (N uint8) -- CUDA tensors, in place."""
        import torch

        n = rung.numel()
        _check(load().fmm_kick_drift(self.h, _ptr(pos, torch.float64, 3 * n, "pos"),
                                     _ptr(vel, torch.float64, 3 * n, "vel"), _ptr(acc, torch.float32, 3 * n, "acc"),
                                     _ptr(rung, torch.uint8, n, "rung"),
                                     _ptr(active_next, torch.uint8, n, "active_next"), n, float(eps), float(dt0),
                                     int(max_rung), int(substep), int(closing)))

    def set_fixed_sources(self, pos, mass, rung=None, r_fixed=0, vel=None, dt=0.0):
        """Fixed tree of the dual-tree scheme: the particles with rung <= r_fixed (all when rung is
        None) at pos + vel * dt (pos when vel is None).  CUDA tensors of the full particle set."""
        import torch

        n = mass.numel()
        _check(load().fmm_set_fixed_sources(self.h, _ptr(pos, torch.float64, 3 * n, "pos"),
                                            _ptr(vel, torch.float64, 3 * n, "vel", True),
                                            _ptr(mass, torch.float32, n, "mass"),
                                            _ptr(rung, torch.uint8, n, "rung", True), n, int(r_fixed), float(dt)))

    def compute_forces_dual(self, pos, mass, eps, theta, acc, pot=None, active=None):
        """Forces on the sinks in active (every particle outside the fixed set when None) from all
        particles: the fixed set as kept by set_fixed_sources, the others at pos.  acc/pot are
        written for the sinks only; n must be the fixed set's."""
        import torch

        n = mass.numel()
        _check(load().fmm_compute_forces_dual(self.h, _ptr(pos, torch.float64, 3 * n, "pos"),
                                              _ptr(mass, torch.float32, n, "mass"),
                                              _ptr(active, torch.uint8, n, "active", True), n, float(eps),
                                              float(theta), _ptr(acc, torch.float32, 3 * n, "acc"),
                                              _ptr(pot, torch.float32, n, "pot", True)))

    def assign_rungs(self, acc, rung, eps, dt0, max_rung):
        """fmm_assign_rungs: rung = the smallest r <= max_rung with dt0 / 2^r <= 0.2 sqrt(eps / |a|)
        (Sec. 3.2).  acc (3N float32), rung (N uint8 out) -- CUDA tensors."""
        import torch

        n = rung.numel()
        _check(load().fmm_assign_rungs(self.h, _ptr(acc, torch.float32, 3 * n, "acc"),
                                       _ptr(rung, torch.uint8, n, "rung"), n, float(eps), float(dt0),
                                       int(max_rung)))

    def stats(self) -> dict:
        """fmm_get_stats of the last solve (pair counts, phase times, launches) as a dict."""
        s = fmm_stats()
        _check(load().fmm_get_stats(self.h, C.byref(s)))
        return s.as_dict()

    # -- learned criterion
    MLP_NP = 8989
    MLP_NW = 8961

    def mlp_load(self, params):
        """fmm_mlp_load: the learned criterion's FMM_MLP_NP parameters (host float32)."""
        p = np.ascontiguousarray(params, dtype=np.float32)
        _check(load().fmm_mlp_load(self.h, p.ctypes.data, p.size))

    def mlp_get(self):
        """fmm_mlp_get: the learned criterion's parameters (host float32 array)."""
        p = np.zeros(self.MLP_NP, np.float32)
        _check(load().fmm_mlp_get(self.h, p.ctypes.data, p.size))
        return p

    def mlp_predict(self, feats):
        """fmm_mlp_predict: predicted log10 error for feature rows feats (n x 8 float32, CUDA)."""
        import torch

        n = feats.shape[0]
        out = torch.zeros(n, dtype=torch.float32, device=feats.device)
        _check(load().fmm_mlp_predict(self.h, _ptr(feats, torch.float32, 8 * n, "feats"), n, out.data_ptr()))
        return out

    def mlp_gradient(self, feats, labels):
        """fmm_mlp_gradient: (gradient over the FMM_MLP_NW weights, loss) of 0.5 mean((y - label)^2)."""
        import torch

        n = labels.numel()
        g = np.zeros(self.MLP_NW, np.float32)
        loss = np.zeros(1, np.float32)
        _check(load().fmm_mlp_gradient(self.h, _ptr(feats, torch.float32, 8 * n, "feats"),
                                       _ptr(labels, torch.float32, n, "labels"), n, g.ctypes.data, loss.ctypes.data))
        return g, float(loss[0])

    def mlp_train(self, feats, labels, epochs=30, batch=256, lr=1e-3, seed=1):
        """fmm_mlp_train on labelled rows (CUDA tensors); returns the last epoch's mean loss."""
        import torch

        n = labels.numel()
        loss = np.zeros(1, np.float32)
        _check(load().fmm_mlp_train(self.h, _ptr(feats, torch.float32, 8 * n, "feats"),
                                    _ptr(labels, torch.float32, n, "labels"), n, int(epochs), int(batch), float(lr),
                                    int(seed), loss.ctypes.data))
        return float(loss[0])

    def mlp_audit(self, pos, mass, eps, theta, band_lo, band_hi, acc_ref, max_pairs):
        """Audit walk: (features (n, 8), labels (n,)) as CUDA tensors."""
        import torch

        n = mass.numel()
        feats = torch.zeros(max_pairs * 8, dtype=torch.float32, device=pos.device)
        labels = torch.zeros(max_pairs, dtype=torch.float32, device=pos.device)
        got = C.c_longlong()
        _check(load().fmm_mlp_audit(self.h, _ptr(pos, torch.float64, 3 * n, "pos"),
                                    _ptr(mass, torch.float32, n, "mass"), n, float(eps), float(theta), float(band_lo),
                                    float(band_hi), _ptr(acc_ref, torch.float32, 3 * n, "acc_ref"), int(max_pairs),
                                    feats.data_ptr(), labels.data_ptr(), C.byref(got)))
        m = got.value
        return feats[:8 * m].reshape(m, 8), labels[:m]

    def mlp_audit_pairs(self, n):
        """fmm_mlp_audit_pairs: the last audit's (sink first, sink count, source first, source count)
        as particle ranges in the sorted order."""
        arrs = [np.zeros(max(n, 1), np.int32) for _ in range(4)]
        _check(load().fmm_mlp_audit_pairs(self.h, *[a.ctypes.data for a in arrs], n))
        return [a[:n] for a in arrs]

    # -- introspection (host numpy outputs)
    def tree_info(self):
        """fmm_tree_info: counts of cells, groups and PP / PC / local entries."""
        v = [C.c_longlong() for _ in range(5)]
        _check(load().fmm_tree_info(self.h, *[C.byref(x) for x in v]))
        return dict(zip(("cells", "groups", "pp", "pc", "local"), (x.value for x in v)))

    def export_order(self, n):
        """fmm_export_order: the sort permutation and the sorted Morton keys."""
        perm = np.zeros(n, np.uint32)
        keys = np.zeros(n, np.uint64)
        _check(load().fmm_export_order(self.h, perm.ctypes.data, keys.ctypes.data))
        return perm, keys

    def export_cells(self):
        """fmm_export_cells: the tree's cells (ranges, links, mass, centre, box, b_max, moments)."""
        nc = self.tree_info()["cells"]
        d = dict(first=np.zeros(nc, np.int32), count=np.zeros(nc, np.int32), parent=np.zeros(nc, np.int32),
                 child=np.zeros(2 * nc, np.int32), nact=np.zeros(nc, np.int32), mass=np.zeros(nc),
                 com=np.zeros(3 * nc), lo=np.zeros(3 * nc), hi=np.zeros(3 * nc), bmax=np.zeros(nc),
                 moments=np.zeros(44 * nc, np.float32))
        keys = ("first", "count", "parent", "child", "nact", "mass", "com", "lo", "hi", "bmax", "moments")
        _check(load().fmm_export_cells(self.h, *[d[k].ctypes.data for k in keys]))
        d["child"] = d["child"].reshape(nc, 2)
        for k in ("com", "lo", "hi"):
            d[k] = d[k].reshape(nc, 3)
        d["moments"] = d["moments"].reshape(nc, 44)
        return d

    def export_lists(self, kind):
        """fmm_export_lists: (sink cell, source first, source count) of the kind's entries."""
        k = KIND[kind]
        n = C.c_longlong()
        _check(load().fmm_export_lists(self.h, k, C.byref(n), None, None, None, 0))
        m = n.value
        sink, first, count = (np.zeros(max(m, 1), np.int32) for _ in range(3))
        _check(load().fmm_export_lists(self.h, k, C.byref(n), sink.ctypes.data, first.ctypes.data,
                                       count.ctypes.data, m))
        return sink[:m], first[:m], count[:m]

    def compute_forces_i32(self, ipos, mass, eps, theta, acc, pot=None, active=None):
        """fmm_compute_forces_i32: ipos a 3n int32 CUDA tensor holding the uint32 fixed-point
        coordinates (x = u * 2^-32), otherwise as compute_forces."""
        import torch

        n = mass.numel()
        _check(load().fmm_compute_forces_i32(self.h, _ptr(ipos, torch.int32, 3 * n, "ipos"),
                                             _ptr(mass, torch.float32, n, "mass"),
                                             _ptr(active, torch.uint8, n, "active", allow_none=True), n,
                                             float(eps), float(theta), _ptr(acc, torch.float32, 3 * n, "acc"),
                                             _ptr(pot, torch.float32, n, "pot", allow_none=True)))

    def kick_drift_i32(self, ipos, vel, acc, rung, active_next, eps, dt0, max_rung, substep, closing):
        """fmm_kick_drift_i32: fixed-point positions (3n int32 holding uint32) and FP32 velocities
        (3n float32), updated in place."""
        import torch

        n = rung.numel()
        _check(load().fmm_kick_drift_i32(self.h, _ptr(ipos, torch.int32, 3 * n, "ipos"),
                                         _ptr(vel, torch.float32, 3 * n, "vel"), _ptr(acc, torch.float32, 3 * n, "acc"),
                                         _ptr(rung, torch.uint8, n, "rung"),
                                         _ptr(active_next, torch.uint8, n, "active_next"), n, float(eps), float(dt0),
                                         int(max_rung), int(substep), 1 if closing else 0))

    def memory_info(self):
        """fmm_memory_info: (device bytes, pinned host bytes) the context holds."""
        d, h = C.c_longlong(), C.c_longlong()
        _check(load().fmm_memory_info(self.h, C.byref(d), C.byref(h)))
        return d.value, h.value

    def debug_walk_capacity(self, scratch_entries=0, list_scale=0):
        """fmm_debug_walk_capacity: the walk's first scratch and list capacities (0: default), a
        test hook that makes the walk overflow and regrow."""
        _check(load().fmm_debug_walk_capacity(self.h, int(scratch_entries), int(list_scale)))

    def debug_local_side(self, min_sinks=-1):
        """fmm_debug_local_side: walks of at least min_sinks sinks (in the context's previous walk)
        run their local expansions on a side stream (0: every walk after the first; negative: the
        default)."""
        _check(load().fmm_debug_local_side(self.h, int(min_sinks)))

    def export_list_shifts(self, kind):
        """fmm_export_list_shifts: the periodic copy (n_x, n_y, n_z) of each entry's source, rows in
        the order of export_lists(kind)."""
        k = KIND[kind]
        n = C.c_longlong()
        _check(load().fmm_export_list_shifts(self.h, k, C.byref(n), None, 0))
        m = n.value
        out = np.zeros(3 * max(m, 1), np.int32)
        _check(load().fmm_export_list_shifts(self.h, k, C.byref(n), out.ctypes.data, m))
        return out[:3 * m].reshape(m, 3)

    def export_walk_levels(self):
        """fmm_export_walk_levels: per level of the walk, the sink cells walked, the checklist
        entries they examined and the most examined by one sink."""
        counts = np.zeros(3 * 256, np.int64)
        nl = C.c_int()
        _check(load().fmm_export_walk_levels(self.h, counts.ctypes.data, 256, C.byref(nl)))
        return counts[:3 * nl.value].reshape(-1, 3)

    def export_locals(self):
        """fmm_export_locals: (group cell, 56 local coefficients) of every group."""
        g = self.tree_info()["groups"]
        cell = np.zeros(max(g, 1), np.int32)
        L = np.zeros(max(g, 1) * 56, np.float32)
        _check(load().fmm_export_locals(self.h, cell.ctypes.data, L.ctypes.data, g))
        return cell[:g], L[:g * 56].reshape(g, 56)
