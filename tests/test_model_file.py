"""The bracket model file (CPU only): format round trip, checksum, the
training domain it carries, and the older format without one."""
import os
import struct
import zlib

import numpy as np
import pytest


def test_committed_model_carries_its_training_domain():
    from paper_2208_09136_gb300 import abi, bracket
    if not os.path.exists(bracket.MODEL_PATH):
        pytest.skip("no trained model file")
    m = bracket.load_model()
    assert m["params"].size == abi.RQA_MLP_PARAMS and np.isfinite(m["params"]).all()
    assert m["domain"] == [(3, 3)]  # the training series are all m = tau = 3
    assert 0.0 < m["tau_lo"] < m["tau_hi"] < 1.0 and m["margin"] >= 0.0


def test_round_trip_and_checksum(tmp_path):
    from paper_2208_09136_gb300 import abi, bracket
    p = np.random.default_rng(0).standard_normal(abi.RQA_MLP_PARAMS).astype(np.float32)
    path = str(tmp_path / "m.bin")
    bracket.save_model(path, p, 0.1, 0.01, 0.99, domain=[(3, 3), (1, 1), (4, 2)])
    m = bracket.load_model(path)
    assert np.array_equal(m["params"], p) and m["domain"] == [(3, 3), (1, 1), (4, 2)]
    raw = bytearray(open(path, "rb").read())
    raw[40] ^= 1  # a bit of the embedding list or the parameters
    open(path, "wb").write(bytes(raw))
    with pytest.raises(ValueError):
        bracket.load_model(path)


def test_first_format_loads_without_a_domain(tmp_path):
    from paper_2208_09136_gb300 import abi, bracket
    p = np.arange(abi.RQA_MLP_PARAMS, dtype=np.float32) * 1e-6
    body = p.tobytes()
    path = str(tmp_path / "v1.bin")
    with open(path, "wb") as f:
        f.write(b"RQAMLP01")
        f.write(struct.pack("<Ifff", p.size, 0.05, 0.005, 0.995))
        f.write(body)
        f.write(struct.pack("<I", zlib.crc32(body) & 0xFFFFFFFF))
    m = bracket.load_model(path)
    assert np.array_equal(m["params"], p) and m["domain"] == []
