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


def test_default_options_new_fields():
    """The options the evaluation scheduling adds: overlapped streams on, leaf-item cost cap
    left to the default / tuning."""
    import paper_1612_04082_gb300 as K
    o = K.kfmm_default_options()
    assert o.streams == 1 and o.eval_item_cost == 0 and o.graphs == 1 and o.autotune == 1
    assert K.PHASES[-3:] == ("tree_split", "tree_lists", "plans")


def test_build_sets_rejects_mismatched_offsets():
    """Offsets are checked on the host before any device work."""
    import numpy as np
    import pytest
    import paper_1612_04082_gb300 as K
    x = np.zeros((10, 3), np.float32)
    with pytest.raises(ValueError):
        K.kfmm_build_sets(None, [0, 5, 10], x, None, [0, 10], x)
    with pytest.raises(ValueError):
        K.kfmm_build_sets(None, [0], x, None, [0], x)


def test_surface_batch_workload():
    """The 32-surface batch: seeded, sizes log-uniform within the stated range, unit normals,
    sets contiguous."""
    import numpy as np
    import workloads as W
    p1, n1, o1 = W.surface_batch(n_sets=8, lo=500, hi=3000)
    p2, n2, o2 = W.surface_batch(n_sets=8, lo=500, hi=3000)
    assert np.array_equal(p1, p2) and np.array_equal(o1, o2)
    sizes = np.diff(o1)
    assert len(sizes) == 8 and o1[0] == 0 and o1[-1] == len(p1)
    assert sizes.min() >= 500 and sizes.max() <= 3000
    assert np.allclose(np.linalg.norm(n1, axis=1), 1.0)


def test_list_entry_decoding_follows_the_header():
    """kifmm_elastic.h: a periodic list item is box | ((9 (sx+1) + 3 (sy+1) + (sz+1)) ^ 13) << 26,
    so the unmoved image is the plain box index; the binding's decoder inverts exactly that."""
    import numpy as np
    import paper_1612_04082_gb300 as K
    rng = np.random.default_rng(0)
    box = rng.integers(0, 1 << 26, 500)
    shift = rng.integers(-1, 2, (500, 3))
    code = 9 * (shift[:, 0] + 1) + 3 * (shift[:, 1] + 1) + (shift[:, 2] + 1)
    items = (box | ((code ^ 13) << 26)).astype(np.int64)
    assert np.all(items < 2 ** 31)  # non-negative int32
    b2, s2 = K.list_entries(items.astype(np.int32))
    assert np.array_equal(b2, box) and np.array_equal(s2, shift)
    b3, s3 = K.list_entries(box.astype(np.int32))
    assert np.array_equal(b3, box) and not np.any(s3)
