"""The C-ABI boundary without a GPU: libibs.so builds and loads, and every
function include/*.h declares is exported by it and bound under the same
name by the Python binding (paper_1410_4803_gb300/ibs.py).  No compute call
is made."""
import ctypes
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DECL = re.compile(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(ibs_[a-z0-9_]+)\s*\(", re.M)


def declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)  # comments may quote calls
        names.update(DECL.findall(text))
    return sorted(names)


def test_header_declares_the_entry_points():
    names = declared()
    for must in ("ibs_init", "ibs_compute", "ibs_compute_batch", "ibs_query", "ibs_ld_r", "ibs_grm",
                 "ibs_cluster_complete", "ibs_shutdown", "ibs_compute_kernel"):
        assert must in names, must
    assert len(names) >= 20


def test_library_exports_every_declared_symbol():
    from paper_1410_4803_gb300 import build
    lib = ctypes.CDLL(build.build_library())
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, f"declared in include/ but not exported: {missing}"


def test_binding_uses_the_same_names():
    src = open(os.path.join(ROOT, "paper_1410_4803_gb300", "ibs.py")).read()
    unbound = [n for n in declared() if f'"{n}"' not in src and f".{n}" not in src]
    assert not unbound, f"declared but not bound in ibs.py: {unbound}"
