"""The FP64 oracle against its pins (CPU only)."""
import pytest

import oracle
from tests import oracle_pins


@pytest.mark.parametrize("check", oracle_pins.ALL_CHECKS, ids=lambda c: c.__name__)
def test_oracle_pin(check):
    check(oracle)


def test_oracle_threads_reported():
    import numpy as np

    A = np.ones((64, 8), np.float32)
    B = np.ones((8, 8), np.float32)
    _, _, used = oracle.gemm(A, B, threads=2)
    assert used >= 1


def test_golden_listing1():
    """The stored 8x5 . 5x16 fixture (Listing 1 shape) equals both the
    oracle and the exact integer product."""
    import json
    import os

    import numpy as np

    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "listing1_8x5x16.json")))
    A = np.array(g["A"], np.float32)
    B = np.array(g["B"], np.float32)
    C0 = np.array(g["C0"], np.float32)
    C, _, _ = oracle.gemm(A, B, g["alpha"], g["beta"], C0)
    assert np.array_equal(C, np.array(g["C"]))
    exact = 1.5 * (A.astype(np.int64) @ B.astype(np.int64)) + 0.5 * C0.astype(np.int64)
    assert np.array_equal(np.array(g["C"]), exact)
