"""The C-ABI library loads and exports every symbol include/soforest.h declares,
and rejects bad arguments on the host before any launch (no GPU needed)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "soforest.h")


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = set(re.findall(r"\b(so_[a-z0-9_]+)\s*\(", txt))
    return sorted(names)


@pytest.fixture(scope="module")
def L():
    from paper_2603_00326_b300 import build, soforest
    build.build()
    return soforest.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("so_split_search", "so_split_search_batch", "so_partition", "so_train_tree"):
        assert required in names


def test_every_declared_symbol_is_exported(L):
    for name in declared_functions():
        assert hasattr(L, name), name


def test_version_and_error_string(L):
    from paper_2603_00326_b300 import soforest as S
    assert "sm_103a" in S.so_version()
    assert isinstance(S.so_last_error(), str)


def _fake_dataset(**kw):
    from paper_2603_00326_b300 import soforest as S
    base = dict(X=0x1000, n=100, d=4, ld=100, y=0x2000, n_classes=2)
    base.update(kw)
    return S.so_dataset(**base)


@pytest.mark.parametrize("kw,what", [
    (dict(n_classes=9), "n_classes"), (dict(n_classes=0), "n_classes"), (dict(ld=50), "ld"),
    (dict(d=0), "d="), (dict(X=0), "NULL"), (dict(n=0), "n="),
])
def test_bad_dataset_rejected_on_host(L, kw, what):
    from paper_2603_00326_b300 import soforest as S
    ds = _fake_dataset(**kw)
    pr = S.so_projs(4, 0x3000, 0x4000, 0x5000)
    prm = S.split_params()
    out = S.so_split()
    st = L.so_split_search(C.byref(ds), C.c_void_p(0x6000), 10, C.byref(pr), C.byref(prm), C.byref(out),
                           None, None, 0, None)
    assert st == S.SO_EINVAL
    assert what in S.so_last_error()


@pytest.mark.parametrize("prm", [dict(n_bins=1), dict(n_bins=257), dict(sort_below=-1), dict(sort_below=5000)])
def test_bad_params_rejected_on_host(L, prm):
    from paper_2603_00326_b300 import soforest as S
    ds = _fake_dataset()
    pr = S.so_projs(4, 0x3000, 0x4000, 0x5000)
    p = S.split_params(**prm)
    out = S.so_split()
    assert L.so_split_search(C.byref(ds), C.c_void_p(0x6000), 10, C.byref(pr), C.byref(p), C.byref(out),
                             None, None, 0, None) == S.SO_EINVAL


def test_bad_projection_header_rejected(L):
    from paper_2603_00326_b300 import soforest as S
    ds = _fake_dataset()
    prm = S.split_params()
    out = S.so_split()
    for pr in (S.so_projs(0, 0x3000, 0x4000, 0x5000), S.so_projs(2000, 0x3000, 0x4000, 0x5000),
               S.so_projs(4, 0, 0x4000, 0x5000)):
        assert L.so_split_search(C.byref(ds), C.c_void_p(0x6000), 10, C.byref(pr), C.byref(prm),
                                 C.byref(out), None, None, 0, None) == S.SO_EINVAL


def test_sampler_and_partition_argument_checks(L):
    from paper_2603_00326_b300 import soforest as S
    assert L.so_sample_projections(4, C.c_void_p(0x10), 8, 10, 1.5, 33, C.c_void_p(0x20), C.c_void_p(0x30),
                                   C.c_void_p(0x40), None) == S.SO_EINVAL
    assert L.so_sample_projections(4, C.c_void_p(0x10), 8, 10, float("nan"), 8, C.c_void_p(0x20),
                                   C.c_void_p(0x30), C.c_void_p(0x40), None) == S.SO_EINVAL
    ds = _fake_dataset()
    nl = C.c_int64(0)
    assert L.so_partition(C.byref(ds), C.c_void_p(0x10), 10, C.c_void_p(0x20), C.c_void_p(0x30), 0,
                          C.c_float(0.0), C.byref(nl), None) == S.SO_EINVAL
    tp = S.tree_params(n_proj=0, lam=1.5, cap=8)
    t = S.so_tree()
    assert L.so_train_tree(C.byref(ds), C.c_void_p(0x10), 10, C.byref(tp), C.byref(t), None) == S.SO_EINVAL


def test_workspace_size_query_is_host_only(L):
    from paper_2603_00326_b300 import soforest as S
    p = S.split_params(n_bins=256, sort_below=1024)
    small = S.so_split_search_ws_bytes(1, 1000, 8, 2, p)
    big = S.so_split_search_ws_bytes(1, 4 << 20, 256, 3, p)
    assert 0 < small < big
    assert big >= 256 * 256 * 3 * 4  # one node's histograms at least


def test_autotune_argument_checks(L):
    from paper_2603_00326_b300 import soforest as S
    ds = _fake_dataset()
    p = S.split_params()
    k = C.c_int32(0)
    for args in ((0, 1.5, 8), (8, -1.0, 8), (8, 1.5, 0), (8, 1.5, 33)):
        assert L.so_autotune(C.byref(ds), args[0], args[1], args[2], C.byref(p), None, None, C.byref(k),
                             None) == S.SO_EINVAL


def test_predict_argument_checks(L):
    from paper_2603_00326_b300 import soforest as S
    f = S.so_forest(1, 2, 8, None, None, None, None, None, None, None, None)
    pred = C.c_int32(0)
    # NULL forest arrays, bad class count, NULL pred: rejected before any launch
    assert L.so_predict(None, 0, 4, 0, C.byref(f), None, C.byref(pred), None) == S.SO_EINVAL
    f2 = S.so_forest(0, 9, 8, None, None, None, None, None, None, None, None)
    assert L.so_predict(None, 0, 4, 0, C.byref(f2), None, C.byref(pred), None) == S.SO_EINVAL
    f3 = S.so_forest(0, 2, 8, None, None, None, None, None, None, None, None)
    assert L.so_predict(None, 0, 4, 0, C.byref(f3), None, None, None) == S.SO_EINVAL
    # an empty forest over zero samples is a no-op
    assert L.so_predict(None, 0, 4, 0, C.byref(f3), None, C.byref(pred), None) == S.SO_OK
