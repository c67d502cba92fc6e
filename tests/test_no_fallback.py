"""The product path has no CPU fallback: a missing CUDA library is an error, host tensors are
refused rather than computed on the host, and nothing in the package imports the oracle."""
import glob
import os
import re

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_missing_library_fails_loudly(tmp_path):
    from paper_1811_06127_gb300 import fmocc
    with pytest.raises(RuntimeError, match="not built"):
        fmocc.load_library(str(tmp_path / "libfmocc.so"))


def test_host_tensors_are_refused():
    from paper_1811_06127_gb300 import fmocc
    with pytest.raises(TypeError, match="CUDA tensor"):
        fmocc._dptr(torch.zeros(4, dtype=torch.int32), fmocc._U32, "k")
    with pytest.raises(TypeError, match="CUDA tensor"):
        fmocc._dptr([0, 1], fmocc._U32, "k")


def test_package_never_imports_the_oracle():
    files = glob.glob(os.path.join(ROOT, "paper_1811_06127_gb300", "**", "*.py"), recursive=True)
    assert files
    pattern = re.compile(r"^\s*(import\s+oracle\b|from\s+oracle\b)", re.M)
    offenders = [f for f in files if pattern.search(open(f).read())]
    assert not offenders, offenders
    # nor does the CUDA source link or include anything of the oracle's
    for f in glob.glob(os.path.join(ROOT, "paper_1811_06127_gb300", "csrc", "*")):
        assert "oracle" not in open(f).read(), f
