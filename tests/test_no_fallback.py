"""The product path has no CPU fallback (CPU only): without the built CUDA
library the binding raises instead of computing, and without a CUDA device
the problem classes refuse to construct."""
import pytest


def test_missing_library_raises(tmp_path, monkeypatch):
    from paper_2304_08232_gb300 import _lib
    monkeypatch.setattr(_lib, "_LIB", None)
    with pytest.raises(ImportError):
        _lib.load(str(tmp_path / "libhpcg_gb300_missing.so"))


def test_no_device_no_problem():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2304_08232_gb300 import HpcgEll, HpcgProblem, HpcgSplit
    for cls in (HpcgProblem, HpcgEll, HpcgSplit):
        with pytest.raises(RuntimeError):
            cls(8, 8, 8, levels=2)


def test_oracle_not_imported_by_the_product_package():
    import pathlib
    root = pathlib.Path(__file__).resolve().parent.parent / "paper_2304_08232_gb300"
    for f in list(root.glob("*.py")) + list((root / "csrc").glob("*")):
        text = f.read_text(errors="ignore")
        assert "import oracle" not in text and "from oracle" not in text and "hpcg_oracle" not in text, f
