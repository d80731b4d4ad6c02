"""CPU-only checks of the C ABI: the library loads, exports every entry point
that include/rqa.h declares, and its host helpers agree with the oracle.
No compute call is made without a GPU."""
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def built():
    from paper_2208_09136_gb300 import build
    return build.build()


def _declared(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rqa_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol(built):
    out = subprocess.run(["nm", "-D", "--defined-only", built], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (rqa_[a-z0-9_]+)", out))
    headers = [h for h in os.listdir(os.path.join(ROOT, "include")) if h.endswith(".h")]
    for h in headers:
        for name in _declared(h):
            assert name in exported, f"{name} declared in {h} but not exported"


def test_binding_resolves_every_symbol(built):
    import paper_2208_09136_gb300 as rqa
    L = rqa.lib()
    for name in _declared("rqa.h"):
        assert hasattr(L, name)
    assert rqa.rqa_abi_version() == 3


@pytest.mark.parametrize("p", [1, 3, 4753, 49975003, 4999350021, (1 << 61) + 12345])
def test_target_counts_match_oracle(built, p):
    import paper_2208_09136_gb300 as rqa
    from oracle import rqa_oracle as O
    for rr, den in [(list(range(1, 21)), 100), ([1, 2, 3, 98, 99], 100), ([1, 5], 7)]:
        got = rqa.rqa_target_counts(p, rr, den)
        assert np.array_equal(got, O.target_counts(p, rr, den))


def test_target_counts_rejects_bad_rates(built):
    import paper_2208_09136_gb300 as rqa
    for rr, den in [([0], 100), ([100], 100), ([-1], 100)]:
        with pytest.raises(rqa.RqaError):
            rqa.rqa_target_counts(1000, rr, den)


def test_error_strings(built):
    import paper_2208_09136_gb300 as rqa
    for code in range(0, 11):
        assert rqa.rqa_error_string(code) != "unknown error"
    assert rqa.rqa_error_string(99) == "unknown error"


def test_create_without_gpu_fails_cleanly(built):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import ctypes
    from paper_2208_09136_gb300 import abi
    p = ctypes.c_void_p()
    cfg = abi._Config(0, None, 0, 0, 0, 0, 0, (ctypes.c_int * 3)())
    rc = abi.lib().rqa_create(ctypes.byref(p), ctypes.byref(cfg))
    assert rc == 4 and not p.value  # RQA_ERR_CUDA, no context


def test_null_context_is_rejected(built):
    from paper_2208_09136_gb300 import abi
    L = abi.lib()
    assert L.rqa_status(None) == 1
    assert L.rqa_eps_for_rr(None, None, None, 100, 20, None, None, None) == 1
    assert L.rqa_det_avg(None, None, None, 100, None, 20, None, 1, None, None, None, None) == 1
    assert L.rqa_line_hist(None, None, None, 20, None, None, None, None, None) == 1
    assert L.rqa_set_timing(None, 1) == 1
    assert L.rqa_kernel_launches(None) == 0


def test_binding_constants_match_header():
    """Every #define of include/rqa.h that the binding mirrors has its value."""
    import paper_2208_09136_gb300.abi as abi
    text = open(os.path.join(ROOT, "include", "rqa.h")).read()
    defines = {k: int(v) for k, v in re.findall(r"#define\s+(RQA_[A-Z0-9_]+)\s+(\d+)", text)}
    mirrored = [k for k in defines if hasattr(abi, k)]
    assert {"RQA_K_MAX", "RQA_FLAG_NO_GRAPHS", "RQA_FLAG_LOI", "RQA_NOALLOC_K_MAX",
            "RQA_NOALLOC_NE_MAX"} <= set(mirrored)
    for k in mirrored:
        assert getattr(abi, k) == defines[k], k


@pytest.mark.parametrize("ne", [2, 11, 100, 101, 4998, 99994, 1 << 31, 1 << 32])
def test_target_counts_loi_match_oracle(built, ne):
    """The identity-line targets (RQA_FLAG_LOI) of the library's host code equal
    the oracle's; rates the identity line reaches alone are rejected by both."""
    import paper_2208_09136_gb300 as rqa
    from oracle import rqa_oracle as O
    for rr, den in [(list(range(1, 100)), 100), ([1, 5, 127], 128), ([1, 2], 3)]:
        try:
            want = O.target_counts_loi(ne, rr, den)
        except ValueError:
            with pytest.raises(rqa.RqaError):
                rqa.rqa_target_counts_loi(ne, rr, den)
            continue
        assert np.array_equal(rqa.rqa_target_counts_loi(ne, rr, den), want)
    with pytest.raises(rqa.RqaError):
        rqa.rqa_target_counts_loi((1 << 32) + 1, [50], 100)


def test_noalloc_rejects_series_beyond_its_item_limit(built):
    """The fixed-scratch entry point checks every size on the host before it
    touches the device: a series with Ne > RQA_NOALLOC_NE_MAX (its work items
    would pass 2^30 cells, beyond what 32-bit shared counts hold exactly) is
    RQA_ERR_CAPACITY, and so is one series too many; an ordinary size gets past
    those checks (to the CUDA calls, which fail here without a GPU)."""
    import ctypes
    import torch
    from paper_2208_09136_gb300 import abi
    if torch.cuda.is_available():
        pytest.skip("a GPU is present: the device path would run")
    L = abi.lib()
    rr = np.arange(1, 21, dtype=np.int32)
    dummy = np.zeros(4, dtype=np.float32)  # never dereferenced: the checks fail first

    def call(lengths, m=1, tau=1):
        offs = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
        ms = np.full(len(lengths), m, dtype=np.int32)
        taus = np.full(len(lengths), tau, dtype=np.int32)
        b = abi._Batch(dummy.ctypes.data, offs.ctypes.data, ms.ctypes.data, taus.ctypes.data,
                       len(lengths))
        return L.rqa_eps_for_rr_noalloc(ctypes.byref(b), rr.ctypes.data, 100, 20,
                                        ctypes.c_void_p(dummy.ctypes.data), None, None, None, None)

    ne_max = abi.RQA_NOALLOC_NE_MAX
    assert call([ne_max + 1]) == 7                 # RQA_ERR_CAPACITY
    assert call([100, ne_max + 3], m=3, tau=1) == 7  # Ne = ne_max + 1 in the second series
    assert call([100] * (abi.RQA_NOALLOC_MAX_SERIES + 1)) == 7
    assert call([ne_max]) == 4                     # accepted sizes reach the device: RQA_ERR_CUDA
