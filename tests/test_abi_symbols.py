"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/*.h (no compute call: this runs without a GPU)."""
import ctypes
import glob
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names.update(re.findall(r"\b(donof_(?:ri|mlp)_\w+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2012_15662_gb300 import binding, build
    if not os.path.exists(binding.LIB_PATH):
        if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
            pytest.skip("nvcc unavailable")
        build.build()
    return ctypes.CDLL(binding.LIB_PATH)


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("donof_ri_init", "donof_ri_transform", "donof_ri_jk_mo", "donof_ri_jk_ao_batch",
                     "donof_ri_energy_lagrangian", "donof_ri_destroy", "donof_ri_strerror"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2012_15662_gb300 import binding
    names = _declared()
    assert names
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) <= set(binding.EXPORTS) | set(names)
    for n in binding.EXPORTS:
        assert n in names, f"binding exports {n} which the header does not declare"


def test_strerror_without_gpu(lib):
    lib.donof_ri_strerror.restype = ctypes.c_char_p
    assert lib.donof_ri_strerror(0) == b"ok"
    assert b"positive definite" in lib.donof_ri_strerror(-4)


def test_init_rejects_bad_arguments_without_gpu(lib):
    from paper_2012_15662_gb300 import binding
    binding.load()
    out = ctypes.c_void_p()
    assert binding.load().donof_ri_init(None, 0, None, ctypes.byref(out)) == binding.DONOF_RI_E_ARG


def test_built_for_sm_103a_only():
    from paper_2012_15662_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
