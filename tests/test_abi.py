"""The C-ABI library builds, loads and exports every entry point include/lamg.h declares
(no compute call: these run without a GPU)."""
import ctypes
import os
import re
import subprocess

import numpy as np

import oracle
import paper_2606_24791_b300 as lamg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "lamg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lamg_\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared()
    for must in ["lamg_setup", "lamg_solve", "lamg_solve_batch", "lamg_serve"]:
        assert must in names


def test_library_exports_every_declared_symbol():
    path = lamg.lib_path()
    lamg.lib()
    assert os.path.exists(path)
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s(lamg_\w+)", out))
    missing = [n for n in declared() if n not in exported]
    assert not missing, missing
    dll = ctypes.CDLL(path)
    for n in declared():
        assert hasattr(dll, n)


def test_options_defaults_are_the_papers():
    o = lamg.options()
    assert (o.K, o.nu_tv, o.dmax, o.nu_pre, o.nu_post) == (4, 3, 4, 1, 2)
    assert o.Q == 2.5 and o.tau_soc == 0.05 and o.veto == 1 and o.caliber2 == 1
    assert ctypes.sizeof(lamg.Options) == 144   # the layout include/lamg.h states
    assert ctypes.sizeof(lamg.SolveOpts) == 32
    assert o.tv_order == lamg.TV_STRIDED == 0 and lamg.TV_STORED == 1
    # the readings' defaults, as include/lamg.h documents them: coarsest size by rule (0), dense
    # small levels up to 4096 nodes, Chebyshev above 32 colours with degree 1, no timing trials,
    # and the oracle's defaults agree wherever both have the option
    assert (o.coarsest_max, o.dense_rows, o.cheb_colours, o.cheb_degree, o.autotune) == (0, 4096, 32, 1, 0)
    for key in ("K", "nu_tv", "dmax", "nu_pre", "nu_post", "coarsest_max", "dense_rows", "cheb_colours",
                "cheb_degree"):
        assert oracle.DEFAULTS[key] == getattr(o, key), key


def test_strerror_names_codes():
    L = lamg.lib()
    assert L.lamg_strerror(0) == b"ok"
    assert b"connected" in L.lamg_strerror(2)


def test_binding_has_no_cpu_fallback():
    # The binding is argument marshalling only: it imports neither the oracle nor numpy/scipy
    # solvers for compute.
    src = open(os.path.join(ROOT, "paper_2606_24791_b300", "__init__.py")).read()
    assert "oracle" not in src.replace("no CPU fallback", "")
    assert "scipy" not in src
