"""The C ABI library builds, loads and exports every entry point declared in
include/surfmcmc.h; host-only calls behave as documented (no GPU needed)."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "surfmcmc.h")


def _declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\**\s*(surfmcmc_\w+)\s*\(", txt, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_1302_2669_gb300 import build as b
    b.build()
    import paper_1302_2669_gb300 as pkg
    return pkg.lib()


def test_header_declares_entry_points():
    names = _declared()
    for n in ("surfmcmc_create", "surfmcmc_destroy", "surfmcmc_decode", "surfmcmc_decode_ex",
              "surfmcmc_gen_syndromes", "surfmcmc_start_frames", "surfmcmc_strerror"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    import paper_1302_2669_gb300 as pkg
    out = subprocess.run(["nm", "-D", "--defined-only", pkg.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\s[TW]\s+(\w+)$", out, flags=re.M))
    for name in _declared():
        assert name in exported, name
        assert hasattr(lib, name)
    assert set(pkg.EXPORTS) <= set(_declared())


def test_host_only_calls(lib):
    import paper_1302_2669_gb300 as pkg
    o = pkg._Opts()
    lib.surfmcmc_default_opts(C.byref(o))
    assert (o.n_classes, o.chains_per_class, o.n_sweeps, o.burn_in, o.beta_scale) == (4, 4, 2000, 0, 1.0)
    for code in (0, -1, -2, -3, -4):
        assert lib.surfmcmc_strerror(code)
    assert lib.surfmcmc_last_error(None) == b""
    # NULL context / out pointer -> EINVAL, without touching a device
    assert lib.surfmcmc_create(None, 0) == pkg.EINVAL
    assert lib.surfmcmc_decode(None, None, 0, 5, 0.1, None, 0, 0, None, None, None, None) == pkg.EINVAL
    lib.surfmcmc_destroy(None)


def test_create_without_device_reports_enodev(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_1302_2669_gb300 as pkg
    h = C.c_void_p()
    assert lib.surfmcmc_create(C.byref(h), 0) == pkg.ENODEV
    assert not h
