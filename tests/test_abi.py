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


@pytest.mark.parametrize("prm", [dict(n_bins=1), dict(n_bins=257), dict(sort_below=-1), dict(sort_below=5000),
                                 dict(bin_rule=2), dict(bin_rule=1), dict(criterion=2), dict(criterion=-1),
                                 dict(proj_per_cta=-1), dict(proj_per_cta=65), dict(chunk=100),
                                 dict(chunk=20000)])
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


def test_struct_layouts_match_header(tmp_path):
    """Every ABI struct of the binding has the C header's size and field
    offsets (compiled here with the host C compiler)."""
    import os
    import shutil
    import subprocess
    from paper_2603_00326_b300 import soforest as S
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    structs = {"so_dataset": S.so_dataset, "so_projs": S.so_projs, "so_split_params": S.so_split_params,
               "so_split": S.so_split, "so_tree_params": S.so_tree_params, "so_tree": S.so_tree,
               "so_forest": S.so_forest, "so_profile_entry": S.so_profile_entry}
    lines = ["#include <stdio.h>", "#include <stddef.h>", "#include \"soforest.h\"", "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for fname, _ in cls._fields_:
            cname = "lambda" if fname == "lambda_" else fname
            lines.append(f'  printf("{name} {fname} %zu\\n", offsetof({name}, {cname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", inc, str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        a, b, v = line.split()
        got[(a, b)] = int(v)
    for name, cls in structs.items():
        assert got[(name, "size")] == C.sizeof(cls), name
        for fname, _ in cls._fields_:
            assert got[(name, fname)] == getattr(cls, fname).offset, (name, fname)


def test_too_small_caller_workspace_is_rejected_on_host(L):
    """A caller workspace below the size the search needs returns SO_ENOMEM
    before any launch, for the one-node and the batched search."""
    from paper_2603_00326_b300 import soforest as S
    ds = _fake_dataset()
    pr = S.so_projs(4, 0x3000, 0x4000, 0x5000)
    prm = S.split_params(n_bins=256, sort_below=0, hist_only=True)
    out = S.so_split()
    need = S.so_split_search_ws_bytes(1, 10, 4, 2, prm)
    assert need > 1024
    for ws in (1, need // 4):
        st = L.so_split_search(C.byref(ds), C.c_void_p(0x6000), 10, C.byref(pr), C.byref(prm), C.byref(out),
                               None, C.c_void_p(0x7000), ws, None)
        assert st == S.SO_ENOMEM, st
        assert "workspace" in S.so_last_error()
        st = L.so_split_search_batch(C.byref(ds), C.c_void_p(0x6000), 10, C.c_void_p(0x6100), 1, C.byref(pr),
                                     C.byref(prm), C.c_void_p(0x6200), None, C.c_void_p(0x7000), ws, None)
        assert st == S.SO_ENOMEM, st
        assert "workspace" in S.so_last_error()


def test_noalloc_shares_the_argument_checks(L):
    """The allocation-free entry point rejects what so_split_search rejects,
    with the same messages, before touching the device."""
    from paper_2603_00326_b300 import soforest as S
    pr = S.so_projs(4, 0x3000, 0x4000, 0x5000)
    out = S.so_split()
    for ds, prm, what in ((_fake_dataset(n_classes=9), S.split_params(), "n_classes"),
                          (_fake_dataset(), S.split_params(n_bins=257), "n_bins"),
                          (_fake_dataset(), S.split_params(bin_rule=1), "bin_keys"),
                          (_fake_dataset(), S.split_params(chunk=100), "chunk")):
        st = L.so_split_search_noalloc(C.byref(ds), C.c_void_p(0x6000), 10, C.byref(pr), C.byref(prm),
                                       C.byref(out), None, None)
        assert st == S.SO_EINVAL
        assert what in S.so_last_error()
    big = S.so_projs(1024, 0x3000, 0x4000, 0x5000)
    st = L.so_split_search_noalloc(C.byref(_fake_dataset(n_classes=8)), C.c_void_p(0x6000), 4000, C.byref(big),
                                   C.byref(S.split_params(256, 0, True)), C.byref(out), None, None)
    assert st == S.SO_EINVAL and "static" in S.so_last_error()


@pytest.mark.parametrize("kw,n_root,root,what", [
    (dict(n_proj=0), 10, 0x7000, "n_proj"), (dict(n_proj=1025), 10, 0x7000, "n_proj"),
    (dict(cap=0), 10, 0x7000, "nnz_cap"), (dict(cap=33), 10, 0x7000, "nnz_cap"),
    (dict(lam=-1.0), 10, 0x7000, "lambda"), (dict(lam=float("nan")), 10, 0x7000, "lambda"),
    (dict(lam=float("inf")), 10, 0x7000, "lambda"),
    (dict(n_bins=1), 10, 0x7000, "n_bins"), (dict(sort_below=5000), 10, 0x7000, "sort_below"),
    (dict(), 0, 0x7000, "n_root"), (dict(), 10, 0, "root_idx"),
])
def test_tree_argument_checks(L, kw, n_root, root, what):
    """so_train_tree rejects its parameters on the host, before any launch."""
    from paper_2603_00326_b300 import soforest as S
    ds = _fake_dataset()
    base = dict(n_proj=8, lam=1.5, cap=8)
    base.update(kw)
    tp = S.tree_params(base.pop("n_proj"), base.pop("lam"), base.pop("cap"), **base)
    out = S.so_tree()
    st = L.so_train_tree(C.byref(ds), C.c_void_p(root), n_root, C.byref(tp), C.byref(out), None)
    assert st == S.SO_EINVAL
    assert what in S.so_last_error()
