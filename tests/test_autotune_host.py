"""Host logic of the batched-GMRES autotuner (no GPU): the fastest shape is chosen
per lane-group width from the per-launch times, written to the JSON cache, and a
second call with the same groups reads the cache instead of timing."""
import json
import types

import pytest


class _FakeSolver:
    calls = 0

    def __init__(self, contexts, warps, ctas_per_sm, reg_budget, **kw):
        self.shape = (warps[0], ctas_per_sm[0], reg_budget[0])

    def solve(self, bs, xs):
        _FakeSolver.calls += 1
        w, c, rb = self.shape
        # width 8 prefers (4, 0, 2), width 32 prefers (8, 0, 1); width 16 absent
        t8 = 1.0 if (w, rb) == (4, 2) else 2.0 + w
        t32 = 3.0 if (w, rb) == (8, 1) else 5.0 + w
        return {"launch_ms": [t8, 0.0, t32]}


@pytest.fixture
def tuner(monkeypatch):
    import torch
    from paper_1704_04549_gb300 import autotune, batch
    monkeypatch.setattr(torch.cuda, "get_device_name", lambda d=None: "FakeGPU")
    monkeypatch.setattr(batch, "BatchGmres", _FakeSolver)
    _FakeSolver.calls = 0
    return autotune


def _ctx(dim, n):
    return types.SimpleNamespace(dim=dim, n=n, device="cuda:0")


def test_pick_per_width_and_cache_round_trip(tuner, tmp_path):
    path = str(tmp_path / "tune.json")
    ctxs = [_ctx(2, 5), _ctx(3, 7), _ctx(2, 24)]
    r1 = tuner.tune_batch_gmres(ctxs, None, None, cache_path=path)
    assert not r1["cached"] and len(r1["table"]) == len(tuner.CANDIDATES)
    assert r1["warps"] == (4, 0, 8) and r1["reg_budget"] == (2, 0, 1)
    calls = _FakeSolver.calls
    assert calls == 2 * len(tuner.CANDIDATES)          # warm-up + timed solve each
    cache = json.load(open(path))
    assert len(cache) == 2 and all(k.startswith("FakeGPU|fp64|m20|") for k in cache)
    r2 = tuner.tune_batch_gmres(ctxs, None, None, cache_path=path)
    assert r2["cached"] and _FakeSolver.calls == calls
    assert (r2["warps"], r2["reg_budget"]) == (r1["warps"], r1["reg_budget"])
    # another precision or another group mix is a different key: timed again
    tuner.tune_batch_gmres(ctxs, None, None, cache_path=path, mixed=True)
    assert _FakeSolver.calls == 2 * calls
    tuner.tune_batch_gmres(ctxs[:1], None, None, cache_path=path)   # 8 lanes: {2d5} only
    assert _FakeSolver.calls == 3 * calls
    tuner.tune_batch_gmres(ctxs[:2] + [_ctx(2, 24)], None, None, cache_path=path)
    assert _FakeSolver.calls == 3 * calls                               # same keys: cached
