"""The C-ABI library builds, loads and exports every function include/*.h declares.
No compute call is made here (this runs without a GPU)."""
import ctypes
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b([a-z]\w*)\s*\(", txt, flags=re.M):
            if not m.group(0).lstrip().startswith(("typedef", "#")):
                names.add(m.group(1))
    return sorted(names)


def test_library_exports_declared_symbols():
    import __graft_entry__
    path = __graft_entry__._build_module().build()
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert len(names) >= 10, names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_helpers():
    import paper_1612_04082_gb300 as K
    o = K.kfmm_default_options()
    assert (o.p, o.leaf_cap) == (6, 64)
    assert K.kfmm_status_str(K.KFMM_ERR_NOT_BUILT) == "not built"
    assert abs(K.material_K(1.0, 0.3) - 13.0 / 6.0) < 1e-14
