"""The autotuner's JSON cache (CPU): the first call times (here a stand-in
for so_autotune) and stores the choices under the GPU model and workload
shape; the same key is served from the file; another shape times again."""
import json

import numpy as np


def test_autotune_cache_round_trip(tmp_path, monkeypatch):
    import torch
    from paper_2603_00326_b300 import soforest as S
    calls = []

    def fake(ds, n_proj, lam, cap, params, stream=None):
        calls.append(n_proj)
        params.sort_below, params.proj_per_cta, params.chunk = 192, 32, 8192
        return params, np.zeros(0), np.zeros((0, 2))

    monkeypatch.setattr(S, "so_autotune", fake)
    X = torch.zeros((8, 100), dtype=torch.float32)
    y = torch.zeros(100, dtype=torch.uint8)
    ds = S.DeviceDataset(X, y, 2)
    path = str(tmp_path / "tune.json")
    p1, cached1 = S.autotune_cached(ds, 16, 1.5, 8, S.split_params(256, 1024, False), cache_path=path)
    assert not cached1 and calls == [16]
    assert (p1.sort_below, p1.proj_per_cta, p1.chunk) == (192, 32, 8192)
    p2, cached2 = S.autotune_cached(ds, 16, 1.5, 8, S.split_params(256, 1024, False), cache_path=path)
    assert cached2 and calls == [16] and (p2.sort_below, p2.proj_per_cta, p2.chunk) == (192, 32, 8192)
    _, cached3 = S.autotune_cached(ds, 24, 1.5, 8, S.split_params(256, 1024, False), cache_path=path)
    assert not cached3 and calls == [16, 24]
    table = json.load(open(path))
    assert len(table) == 2 and all(v["chunk"] == 8192 for v in table.values())


def test_autotune_cache_ignores_an_older_procedure(tmp_path, monkeypatch):
    """Choices stored by an older tuning procedure (another version in the
    key) are timed again, not served."""
    import torch
    from paper_2603_00326_b300 import soforest as S
    calls = []

    def fake(ds, n_proj, lam, cap, params, stream=None):
        calls.append(n_proj)
        params.sort_below, params.proj_per_cta, params.chunk = 192, 32, 4096
        return params, np.zeros(0), np.zeros((0, 2))

    monkeypatch.setattr(S, "so_autotune", fake)
    X = torch.zeros((8, 100), dtype=torch.float32)
    y = torch.zeros(100, dtype=torch.uint8)
    ds = S.DeviceDataset(X, y, 2)
    prm = S.split_params(256, 1024, False)
    key = S._autotune_key(ds, 16, 1.5, 8, prm, "cpu")
    assert key.startswith(f"v{S.AUTOTUNE_VERSION}|")
    old_key = "v1|" + key.split("|", 1)[1]
    path = tmp_path / "tune.json"
    path.write_text(json.dumps({old_key: {"sort_below": 64, "proj_per_cta": 16, "chunk": 16384}}))
    p, cached = S.autotune_cached(ds, 16, 1.5, 8, prm, cache_path=str(path))
    assert not cached and calls == [16] and (p.sort_below, p.proj_per_cta, p.chunk) == (192, 32, 4096)
