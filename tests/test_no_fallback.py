"""The product path has no CPU fallback: a copy of the package without its
built library refuses to import, instead of counting some other way."""
import os
import shutil
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_import_without_library_fails(tmp_path):
    dst = tmp_path / "paper_2210_00389_gb300"
    shutil.copytree(os.path.join(ROOT, "paper_2210_00389_gb300"), dst,
                    ignore=shutil.ignore_patterns("*.so", "__pycache__", "_build*"))
    assert not (dst / "libcetc.so").exists()
    out = subprocess.run([sys.executable, "-c", "import paper_2210_00389_gb300"],
                         cwd=tmp_path, capture_output=True, text=True, timeout=120)
    assert out.returncode != 0
    assert "ImportError" in out.stderr and "libcetc.so" in out.stderr
