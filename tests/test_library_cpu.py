"""CPU checks of the C ABI boundary: the CUDA library builds for sm_103a, loads, and exports
every entry point declared in include/nlfeti.h (no compute call is made without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "nlfeti.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(nlfeti_[a-z_]+)\s*\(", src)))


def test_header_declares_the_abi():
    names = declared_symbols()
    for n in ["nlfeti_create", "nlfeti_problem_create", "nlfeti_factor", "nlfeti_solve", "nlfeti_submit",
              "nlfeti_wait", "nlfeti_get_decomposition", "nlfeti_apply"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2306_00094_gb300 import binding
    path = binding._build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_symbols() if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(binding.EXPORTED) == declared_symbols()


def test_default_options_without_gpu():
    from paper_2306_00094_gb300 import binding
    o = binding.default_options()
    assert o.precision == 0 and o.tol == 1e-10 and o.batched == 1


def test_context_fails_loudly_without_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2306_00094_gb300 import binding
    with pytest.raises(binding.NlfetiError):
        binding.Context()
