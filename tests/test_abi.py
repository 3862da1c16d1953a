"""The C-ABI library loads without a GPU and exports every entry point that
``include/*.h`` declares."""
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"^\s*(?:const\s+)?[\w ]+?\**\s*\b(mg_\w+)\s*\(", src, flags=re.M))
    return names


def test_header_declares_the_boundary():
    names = declared()
    for n in ("mg_init", "mg_setup", "mg_solve", "mg_vcycle", "mg_submit", "mg_poll", "mg_free", "mg_destroy"):
        assert n in names


def test_library_loads_and_exports_all_symbols():
    from paper_2405_05047_gb300 import binding
    from paper_2405_05047_gb300 import build
    path = build.build()
    binding.load_library(path)
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (mg_\w+)", out))
    missing = declared() - exported
    assert not missing, missing


def test_no_gpu_raises_cleanly():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    import paper_2405_05047_gb300 as G
    with pytest.raises(G.MGError):
        G.Context(0)
