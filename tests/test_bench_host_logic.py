"""bench.py's orchestration of the Table 2 sweep on the CPU: the library and the CUDA events
replaced by stand-ins that return fixed sizes, so that only the host logic runs (the
per-column keys, alpha = N_over / N, m = nnz / N, the grids and aspect ratios)."""
import types

import numpy as np
import pytest


class _Event:
    def __init__(self, enable_timing=False):
        self.t = 0.0

    def record(self, stream=None):
        pass

    def elapsed_time(self, other):
        return 2.0   # ms


class _Corr:
    def __init__(self, n):
        self.n = n

    def info(self):
        return 100 * self.n, 3 * self.n   # nnz, N_over

    def close(self):
        pass


class _Near:
    def close(self):
        pass


def test_table2_sweep_host_logic(monkeypatch):
    import torch

    import bench
    from paper_2006_02545_gb300 import workloads as W
    monkeypatch.setattr(torch.cuda, "Event", _Event)
    monkeypatch.setattr(W, "TABLE2_GRIDS", ((3, 4), (4, 3)))
    fake = types.SimpleNamespace(
        DeviceSurface=lambda deg, off, xyz: types.SimpleNamespace(n=int(off[-1])),
        params=lambda eps, **kw: types.SimpleNamespace(eps=eps),
        build_near_lists=lambda ctx, ds, x, tn, p: _Near(),
        gen_corrections=lambda ctx, ds, near, kind, k, p: _Corr(ds.n))
    ctx = types.SimpleNamespace(sync=lambda *a: 0, stage_times=lambda: (np.zeros(6), 0))
    rows = bench.table2_sweep(ctx, fake, W, "cpu", None, torch.empty(4))
    assert [r["column"] for r in rows] == [1, 2]
    assert [r["grid"] for r in rows] == [[3, 4], [4, 3]]
    for r, (n_u, n_v) in zip(rows, ((3, 4), (4, 3))):
        assert r["patches"] == 2 * n_u * n_v and r["points"] == 10 * r["patches"]   # degree 3
        assert r["alpha"] == pytest.approx(3.0) and r["m"] == pytest.approx(100.0)
        assert r["S_init"] == pytest.approx(r["points"] / 2e-3)
        assert r["status"] == 0 and len(r["stages_ms"]) == 6
        assert r["a_avg"] >= 1.0
