"""The C-ABI library builds, loads and exports every entry point that
include/am.h declares; argument checks that need no GPU behave as stated."""
import ctypes
import os
import re

import pytest

from paper_2107_10800_gb300 import build, binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build.build()
    return binding.lib()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "am.h")).read()
    return sorted(set(re.findall(r"AM_API\s+[\w\s\*]+?\b(am_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("am_create", "am_set_bodies", "am_set_constraints", "am_solve_step",
                     "am_destroy"):
        assert required in names


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(L, name), name
        assert name in binding.SIGNATURES, name


def test_only_am_symbols_exported():
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", binding.LIB_PATH],
                         capture_output=True, text=True).stdout
    funcs = [l.split()[-1] for l in out.splitlines() if " T " in l]
    assert funcs and all(f.startswith("am_") for f in funcs), funcs


def test_flop_counts(L):
    assert binding.flops_per_pair(0) == 35
    assert binding.flops_per_pair(1) > binding.flops_per_pair(0)


def test_create_rejects_bad_config(L):
    bad = [dict(eta=0.0), dict(a=-1.0), dict(wall=2), dict(tol=0.0), dict(restart=500)]
    for kw in bad:
        args = dict(eta=1.0, a=0.1, wall=0, precision=0, n_systems=1, tol=1e-8, restart=50,
                    max_iter=100, corr_tol=1e-10, corr_max_iter=10, cuda_stream=None)
        args.update({"blob_radius" if k == "a" else k: v for k, v in kw.items()})
        args.pop("a", None)
        cfg = binding.Config(args["eta"], args.get("blob_radius", 0.1), args["wall"],
                             args["precision"], args["n_systems"], args["tol"], args["restart"],
                             args["max_iter"], args["corr_tol"], args["corr_max_iter"], None)
        h = ctypes.c_void_p()
        assert L.am_create(ctypes.byref(cfg), ctypes.byref(h)) == binding.AM_ERR_ARG
        assert not h.value


def test_matvec_argument_checks(L):
    assert L.am_rpy_matvec(None, None, None, -1, 1.0, 0.1, 0, 0, None, 0, None) == binding.AM_ERR_ARG
    assert L.am_rpy_matvec(None, None, None, 0, 1.0, 0.1, 0, 0, None, 0, None) == binding.AM_OK
    assert L.am_rpy_matvec(None, None, None, 10, 0.0, 0.1, 0, 0, None, 0, None) == binding.AM_ERR_ARG
    assert L.am_rpy_matvec(None, None, None, 10, 1.0, 0.1, 0, 7, None, 0, None) == binding.AM_ERR_ARG
    assert b"precision" in L.am_last_error(None)
    assert L.am_rpy_matvec_workspace(0, 0) == 0
    assert L.am_rpy_matvec_workspace(1000, 0) >= 1000 * 32 + 1000 * 24


def test_null_handle_is_rejected(L):
    assert L.am_solve(None, None, None, None, None) == binding.AM_ERR_ARG
    assert L.am_set_initial_guess(None, 1) == binding.AM_ERR_ARG
    L.am_destroy(None)


def test_learned_constants_match_oracle(L):
    from oracle import mlp as om
    text = open(os.path.join(ROOT, "include", "am.h")).read()
    consts = dict(re.findall(r"#define (AM_MLP_\w+) (\d+)", text))
    assert int(consts["AM_MLP_FEAT"]) == om.FEAT == binding.MLP_FEAT
    assert int(consts["AM_MLP_OUT"]) == om.OUT == binding.MLP_OUT
    assert int(consts["AM_MLP_PARAMS"]) == om.n_params() == L.am_mlp_num_params()


def test_learned_argument_checks(L):
    assert L.am_set_learned(None, None, 1) == binding.AM_ERR_ARG
    assert L.am_learned_features(None, None, None) == binding.AM_ERR_ARG
    assert L.am_mlp_create(0, None, None) == binding.AM_ERR_ARG
    assert L.am_mlp_get_params(None, None) == binding.AM_ERR_ARG
    assert L.am_mlp_train(None, None, None, 0, 1, 1, 1e-3, 0, None) == binding.AM_ERR_ARG
    L.am_mlp_destroy(None)


def _struct_fields(name):
    """Field names of a typedef struct in include/am.h, in order."""
    text = open(os.path.join(ROOT, "include", "am.h")).read()
    body = re.search(r"typedef struct \{([^{}]*)\}\s*" + name + ";", text).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    names = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        for part in decl.split(","):
            m = re.search(r"(\w+)\s*(\[\s*\d+\s*\])?\s*$", part.strip())
            names.append(m.group(1))
    return names


def test_binding_structs_mirror_the_header():
    # the ctypes mirrors of am_config and am_step_stats list the header's
    # fields in the header's order (a mismatch would shift every later field)
    assert [f for f, _ in binding.Config._fields_] == _struct_fields("am_config")
    assert [f for f, _ in binding.StepStats._fields_] == _struct_fields("am_step_stats")
