"""The C-ABI library builds for sm_103a, loads, and exports every symbol ufe.h declares."""
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "ufe.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ufe_[a-z_0-9]+)\s*\(", src)))


@pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                    reason="nvcc not available")
def test_library_exports_every_declared_symbol():
    from paper_1703_06323_gb300 import build_ext
    path = build_ext.build()
    from paper_1703_06323_gb300 import ufe
    declared = _declared()
    assert len(declared) >= 20
    for name in declared:
        assert hasattr(ufe.LIB, name), name
    assert set(declared) == set(ufe.EXPORTED)
    assert ufe.ufe_version() == 100
    assert os.path.exists(path)
