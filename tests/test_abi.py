"""The C ABI library: builds, loads and exports every function of include/mine.h.

CPU only: no call here touches a GPU.
"""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_1509_08639_gb300 import _build, mine, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mine.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mine_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    return mine.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ["mine_open", "mine_close", "mine_dict_create", "mine_dict_destroy", "mine_submit",
              "mine_submit_sweep", "mine_poll", "mine_result_free", "mine_align_matrix",
              "mine_run_batch", "mine_run_batch_device"]:
        assert f in names


def test_library_exports_every_declared_function(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", _build.LIB], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r" T (mine_[a-z0-9_]+)$", out, flags=re.M))
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, missing
    # and the binding knows the signature of each of them
    assert sorted(mine.SIGNATURES) == declared_functions()
    for f in declared_functions():
        assert getattr(lib, f) is not None


def test_build_targets_sm_103a_only():
    assert _build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_batch_capacity_is_host_logic(lib):
    b = synth.workload(2, n_pairs=50).batch
    S, T = b.sizes()
    do = np.ascontiguousarray(b.doc_off)
    for n in (1, 3, 64):
        cap = lib.mine_batch_capacity(ctypes.c_void_p(do.ctypes.data), b.n_pairs, n)
        assert cap == int(n * np.minimum(S, T).sum())


def test_last_error_is_a_string(lib):
    assert isinstance(lib.mine_last_error(), bytes)


def test_null_arguments_are_rejected_without_a_device(lib):
    # argument checks run before any CUDA call
    assert lib.mine_open(None, None) == -1
    assert lib.mine_close(None) == 0
    assert lib.mine_poll(None, None, 0, 0) == -1
    assert lib.mine_dict_create(None, None, None, None, 0, None) == -1
    assert lib.mine_align_matrix(None, None, 0, 0, 0, 0, None, None, None) == -1
    assert lib.mine_run_batch(None, None, None, None, None, None, None, None, 0) == -1
    assert lib.mine_run_batch_async(None, None, None, None, None, None, None, None, 0, None) == -1
    assert lib.mine_batch_wait(None, 1) == -1
    assert lib.mine_check(None) == -1
    assert lib.mine_align_strategy_save(None, None) == -1
    assert lib.mine_align_strategy_load(None, None) == -1
