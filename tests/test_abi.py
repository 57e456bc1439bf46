"""The C-ABI library loads and exports every entry point declared in include/igs.h (CPU)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "igs.h")


def declared():
    hdr = open(HEADER).read()
    return set(re.findall(r"^\s*(?:int|const char\*)\s+(igs_\w+)\s*\(", hdr, re.M))


@pytest.fixture(scope="module")
def lib():
    from paper_1703_10016_gb300 import build
    build.build_library()
    from paper_1703_10016_gb300 import igs
    return igs


def test_every_declared_symbol_is_exported(lib):
    out = subprocess.run(["nm", "-D", lib.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (igs_\w+)", out))
    assert declared() <= exported
    assert set(lib.EXPORTED) == declared()


def test_every_declared_symbol_is_bound(lib):
    for name in declared():
        assert hasattr(lib._lib, name)
        assert hasattr(lib, name)


def test_header_documents_citations():
    hdr = open(HEADER).read()
    for tag in ("Algorithm 1", "Algorithm 2", "eq. IK1e2", "eq. IK1e2_bis", "eq. sistlin", "Sect. 5"):
        assert tag in hdr
