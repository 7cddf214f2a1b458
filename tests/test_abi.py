"""The C-ABI library builds, loads without a GPU and exports every function
include/spider.h declares.  No compute calls."""
import ctypes
import os
import subprocess

import pytest

from paper_2508_12117_gb300 import binding

LIB = binding.LIB_PATH


@pytest.fixture(scope="module")
def lib_path():
    if not os.path.exists(LIB):
        from paper_2508_12117_gb300 import _build
        _build.build()
    return LIB


def test_header_declares_the_boundary():
    names = binding.declared_symbols()
    for n in ("spider_create", "spider_grad_logpost", "spider_sgld_step", "spider_samples",
              "spider_get_state", "spider_set_state", "spider_destroy", "spider_last_error",
              "spider_tt_pairs", "spider_philox_words"):
        assert n in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    missing = [n for n in binding.declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if l.strip()}
    assert set(binding.declared_symbols()) <= exported


def test_binding_signatures_load(lib_path):
    L = binding.load_library(lib_path)
    cfg = binding.config_default()
    assert cfg.thin == 1 and cfg.block_obs == 4096 and abs(cfg.kappa - 0.03) < 1e-12
    # a failing create reports INVAL without touching the device
    h = ctypes.c_void_p()
    rc = L.spider_create(None, None, None, ctypes.byref(cfg), None, ctypes.byref(h))
    assert rc == -1 and not h.value
