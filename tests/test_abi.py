"""The C-ABI library builds, loads, and exports every entry point that
include/lse.h declares (no GPU needed: nothing is computed)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="session")
def lib():
    from paper_1705_06073_gb300 import build, lse
    build.build()
    return lse.load()


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "lse.h")).read()
    return sorted(set(re.findall(r"LSE_API\s+[\w\s\*]*?\b(lse_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("lse_create", "lse_fit", "lse_fit_batch", "lse_eval_grid", "lse_destroy", "lse_strerror"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    import subprocess
    from paper_1705_06073_gb300 import lse
    out = subprocess.run(["nm", "-D", "--defined-only", lse.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s+(lse_\w+)", out))
    missing = [n for n in declared_symbols() if n not in exported]
    assert not missing, missing
    for n in declared_symbols():
        assert hasattr(lib, n)
    assert set(lse.EXPORTS) <= set(declared_symbols())


def test_strerror_needs_no_device(lib):
    from paper_1705_06073_gb300 import lse
    assert "invalid" in lse.lse_strerror(lse.LSE_EINVAL)
    assert lse.lse_strerror(lse.LSE_OK) == "ok"


def test_config_defaults_follow_the_paper(lib):
    from paper_1705_06073_gb300 import lse
    c = lse.lse_config_default()
    assert c.tau == 5.0 and c.max_inner == 5 and c.grid_size == 0 and c.precision == lse.LSE_PREC_FP64
