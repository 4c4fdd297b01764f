"""The device Philox4x32-10 (the generator behind every draw of the library)
against the published known-answer vectors and against the oracle's
Philox on many counters and keys, bit for bit."""
import numpy as np
import pytest

import paper_1704_04362_gb300 as tp
from oracle import philox_ref as P
from tests.test_oracle_sampling import PHILOX_KAT

pytestmark = pytest.mark.gpu


def test_device_philox_known_answer_vectors():
    for ctr, key, want in PHILOX_KAT:
        got = tp.philox4x32_10(np.array([ctr], dtype=np.uint32), *key)
        assert tuple(int(x) for x in got[0]) == want, [hex(int(x)) for x in got[0]]


def test_device_philox_matches_oracle_on_random_counters():
    rng = np.random.default_rng(11)
    n = 100003
    ctr = rng.integers(0, 2 ** 32, size=(n, 4), dtype=np.uint64).astype(np.uint32)
    for k0, k1 in ((0, 0), (12345, 0), (0xdeadbeef, 0x01234567)):
        got = tp.philox4x32_10(ctr, k0, k1)
        ref = np.stack(P.philox4x32_10(ctr[:, 0], ctr[:, 1], ctr[:, 2], ctr[:, 3], k0, k1),
                       axis=1).astype(np.uint32)
        assert np.array_equal(got, ref)


def test_device_philox_empty_and_argument_checks():
    import ctypes
    L = tp.lib()
    assert L.tp_philox4x32_10(None, 0, 0, 0, None, None) == 0
    assert L.tp_philox4x32_10(None, 0, 0, 4, None, None) == -2
    assert L.tp_philox4x32_10(None, 0, 0, -1, None, None) == -1
