"""The C-ABI library builds for sm_103a, loads, and exports every entry point
declared in include/qap.h (no GPU needed: nothing is called)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            with open(os.path.join(ROOT, "include", fn)) as f:
                text = re.sub(r"/\*.*?\*/", "", f.read(), flags=re.S)
            names.update(re.findall(r"\b(qap_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_entry_points():
    names = declared_functions()
    for required in ["qap_create", "qap_destroy", "qap_cost", "qap_2opt", "qap_tabu",
                     "qap_search", "qap_search_async", "qap_strerror"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2307_11248_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_strerror_without_gpu():
    import paper_2307_11248_gb300 as q
    assert q.strerror(q.EINVAL) == "invalid argument"
    assert q.strerror(q.EUNSUPPORTED).startswith("instance outside")


def test_create_rejects_bad_arguments_before_touching_the_gpu():
    import numpy as np
    import paper_2307_11248_gb300 as q
    with pytest.raises(q.QapError) as e:
        q.qap_create(np.zeros((1, 1)), np.zeros((1, 1)))
    assert e.value.status == q.EINVAL
    # B = (n^2 + 8n + 32) max|F| max|D| = 80 * 2^40 * 2^22 >= 2^62: no exact
    # int64 path for it
    F = np.full((4, 4), 1 << 40, dtype=np.int64)
    D = np.full((4, 4), -(1 << 22), dtype=np.int64)
    with pytest.raises(q.QapError) as e:
        q.qap_create(F, D)
    assert e.value.status == q.EOVERFLOW
    F[0, 0] = np.iinfo(np.int64).min  # |F| itself beyond int64
    with pytest.raises(q.QapError) as e:
        q.qap_create(F, np.ones((4, 4), dtype=np.int64))
    assert e.value.status == q.EOVERFLOW
    with pytest.raises(q.QapError) as e:
        q.qap_create(np.zeros((300, 300)), np.zeros((300, 300)))
    assert e.value.status == q.EUNSUPPORTED


def test_best_walks_reduction_on_the_host():
    """The host reduction over walks (lowest cost, ties to the lowest walk
    index) runs without a GPU and agrees with a first-occurrence arg-min."""
    import numpy as np
    import paper_2307_11248_gb300 as q
    rng = np.random.default_rng(3)
    c = rng.integers(0, 5, size=(7, 9)).astype(np.int64)  # many ties
    idx = q.qap_best_walks(c, 9)
    assert idx.tolist() == np.argmin(c, axis=1).tolist()
    assert q.qap_best_walks(np.array([5, 5, 5]), 3).tolist() == [0]
    assert q.qap_best_walks(np.zeros(0, dtype=np.int64), 4).tolist() == []
    with pytest.raises(q.QapError) as e:
        q.qap_best_walks(c, 0)
    assert e.value.status == q.EINVAL
