"""The product path has no CPU fallback and never reaches the oracle (CPU).

Without the built CUDA library every entry point of the binding raises
instead of computing; and no module of the package imports, loads or names
the oracle, which is test infrastructure only.
"""
import ast
import os
import pathlib

import pytest

from paper_2603_00326_b300 import soforest as S

PKG = pathlib.Path(S.__file__).resolve().parent


def test_missing_library_raises(monkeypatch):
    monkeypatch.setattr(S, "_lib", None)
    monkeypatch.setattr(S, "LIB_PATH", os.path.join(str(PKG), "lib", "does_not_exist.so"))
    with pytest.raises(ImportError):
        S.lib()
    with pytest.raises(ImportError):
        S.so_launch_count()
    prm = S.split_params(256, 1024, False)  # a plain struct: building it needs no library
    with pytest.raises(ImportError):
        S.so_split_search_ws_bytes(1, 1000, 8, 2, prm)


def test_package_never_reaches_the_oracle():
    sources = sorted(PKG.rglob("*.py")) + sorted(PKG.rglob("*.cu")) + sorted(PKG.rglob("*.cuh")) + \
        sorted(PKG.rglob("*.h"))
    assert len(sources) > 5
    for path in sources:
        text = path.read_text()
        if path.suffix == ".py":
            tree = ast.parse(text)
            for node in ast.walk(tree):
                if isinstance(node, ast.Import):
                    assert all(not a.name.split(".")[0] == "oracle" for a in node.names), path
                elif isinstance(node, ast.ImportFrom):
                    assert (node.module or "").split(".")[0] != "oracle", path
        assert "so_oracle" not in text and "orc_" not in text, path
