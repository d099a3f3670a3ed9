"""The C ABI: every function declared in include/*.h is exported by the built library, the
library loads without a GPU, and calls that need no device validate their arguments."""
import ctypes as C
import glob
import os
import re
import subprocess

import pytest

from paper_1609_08621_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(fmm_\w+)\s*\(", src):
            names.add(m.group(1))
    return names


def test_library_exports_every_declared_symbol():
    lib = build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True, check=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    decl = declared_functions()
    assert len(decl) >= 15
    missing = decl - exported
    assert not missing, f"declared but not exported: {sorted(missing)}"


def test_library_loads_and_host_only_calls_work():
    L = binding.load()
    p = binding.fmm_default_params()
    assert p.theta == 0.55 and p.bucket == 16 and p.group == 64 and p.terms == 15 and p.nrep == 0
    assert binding.fmm_flops_per_pc() > 200
    loc, mom = binding.fmm_multi_index()
    assert loc.shape == (56, 3) and mom.shape == (32, 3)
    assert sorted(map(tuple, loc.tolist())) == sorted({(a, b, o - a - b) for o in range(6) for a in range(o + 1)
                                                       for b in range(o - a + 1)})
    assert L.fmm_default_params(None) == -1
    assert b"NULL" in L.fmm_last_error()
    # invalid arguments are rejected before any device work
    assert L.fmm_set_params(None, C.byref(p)) == -1
    assert L.fmm_compute_forces(None, None, None, None, 0, 0.1, 0.5, None, None) == -1


def declared_arities():
    out = {}
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        for m in re.finditer(r"\b(fmm_\w+)\s*\(([^)]*)\)", src):
            args = m.group(2).strip()
            out[m.group(1)] = 0 if args in ("", "void") else args.count(",") + 1
    return out


def test_binding_signatures_match_header():
    """Every ctypes prototype of the binding takes as many arguments as the header declares."""
    lib = binding.load()
    for name, k in declared_arities().items():
        f = getattr(lib, name)
        if f.argtypes is not None:
            assert len(f.argtypes) == k, (name, len(f.argtypes), k)


def test_network_sizes_agree():
    from oracle import mlp as omlp

    src = open(os.path.join(ROOT, "include", "fmm.h")).read()
    np_ = int(re.search(r"#define FMM_MLP_NP (\d+)", src).group(1))
    nw = int(re.search(r"#define FMM_MLP_NW (\d+)", src).group(1))
    assert (np_, nw) == (omlp.N_PARAMS, omlp.N_WEIGHTS) == (binding.Context.MLP_NP, binding.Context.MLP_NW)


def test_static_order_limit_agrees():
    src = open(os.path.join(ROOT, "include", "fmm.h")).read()
    assert int(re.search(r"#define FMM_STATIC_ORDER_MAX_N (\d+)", src).group(1)) == binding.STATIC_ORDER_MAX_N
