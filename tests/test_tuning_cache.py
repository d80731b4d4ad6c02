"""The tuning cache on the host (no GPU): its key and the store / reuse cycle,
with the library's tuning calls replaced by fakes."""
import json

import numpy as np


def test_batch_key_classes():
    from paper_2208_09136_gb300 import tuning
    k = tuning.batch_key("GB300", 152, [0, 100, 100_100], [3, 3], [3, 3], 20)
    assert k == "GB300|sm152|n2^17|m3t3|K20"
    assert tuning.batch_key("GB300", 152, [0, 50, 90], [3, 1], [3, 1], 20).endswith("|mixed|K20")
    assert "n2^17" in tuning.batch_key("X", 1, [0, 131072], [1], [1], 5)   # 2^17 exactly
    assert "n2^18" in tuning.batch_key("X", 1, [0, 131073], [1], [1], 5)


def test_tuned_stores_then_reuses(tmp_path, monkeypatch):
    from paper_2208_09136_gb300 import abi, tuning
    calls = {"autotune": 0, "set": []}
    state = {"tile": 16, "unit_bands": 0, "line_ctas": 0, "stage": 0, "ms": 0.0}

    def fake_autotune(ctx, batch, rr, den):
        calls["autotune"] += 1
        state.update(tile=32, unit_bands=4, line_ctas=6, stage=1, ms=1.5)
        return dict(state)

    def fake_set(ctx, tile=0, unit_bands=0, line_ctas=0, stage=0):
        calls["set"].append((tile, unit_bands, line_ctas, stage))
        state.update(tile=tile, unit_bands=unit_bands, line_ctas=line_ctas, stage=stage)

    monkeypatch.setattr(abi, "rqa_autotune", fake_autotune)
    monkeypatch.setattr(abi, "rqa_set_tuning", fake_set)
    monkeypatch.setattr(abi, "rqa_get_tuning", lambda ctx: dict(state))
    monkeypatch.setattr(abi, "rqa_device_info", lambda ctx: {"sm_count": 152, "tile": 16, "blocks_per_sm": 0})

    class FakeBatch:
        offsets = np.array([0, 1000, 3000])
        m = np.array([3, 3])
        tau = np.array([3, 3])

    path = str(tmp_path / "tune.json")
    first = tuning.tuned(None, FakeBatch(), list(range(1, 21)), 100, path=path, gpu_name="GB300")
    assert first["cached"] is False and calls["autotune"] == 1
    assert json.load(open(path))[first["key"]]["tile"] == 32
    state.update(tile=16, unit_bands=0, line_ctas=0, stage=0)
    second = tuning.tuned(None, FakeBatch(), list(range(1, 21)), 100, path=path, gpu_name="GB300")
    assert second["cached"] is True and calls["autotune"] == 1
    assert calls["set"] == [(32, 4, 6, 1)]
