"""The device Philox4x32-10 routine, through the C ABI, against the generator's
published known-answer vectors (tests/golden) and against the oracle's word
streams on the counters the draws of Sec. 3.2 and Sec. 3.3 use."""
import ctypes

import numpy as np
import pytest

import oracle
from kat import philox_kat

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def _device_philox(ctr_key: np.ndarray) -> np.ndarray:
    from paper_2202_00517_gb300 import _lib
    lib = _lib.load()
    ck = torch.from_numpy(ctr_key.astype(np.uint32).view(np.int32).reshape(-1)).cuda()
    out = torch.zeros(ck.numel() // 6 * 4, dtype=torch.int32, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = lib.knnd_philox4x32_10(ctypes.c_void_p(ck.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                ck.numel() // 6, stream)
    assert st == _lib.KNND_OK
    torch.cuda.synchronize()
    return out.cpu().numpy().view(np.uint32).reshape(-1, 4)


def test_device_philox_known_answers():
    rows = philox_kat()
    ck = np.stack([np.concatenate([c, k]) for c, k, _ in rows])
    got = _device_philox(ck)
    for (c, k, want), g in zip(rows, got):
        assert np.array_equal(g, want), (c, k, g, want)


def test_device_philox_matches_oracle_streams():
    """Init-graph counters (x, 0, 0, block) and clustering-sample counters
    (s, r, 1, block) for a 64-bit seed, several blocks each."""
    seed = 0x0123456789ABCDEF
    rows, want = [], []
    for c0, c1, c2 in ((0, 0, 0), (999_999, 0, 0), (17, 3, 1), (9_999, 10, 1)):
        words = oracle.stream_words(seed, c0, c1, c2, 12)
        for blk in range(3):
            rows.append([c0, c1, c2, blk, seed & 0xFFFFFFFF, seed >> 32])
            want.append(words[4 * blk:4 * blk + 4])
    got = _device_philox(np.array(rows, dtype=np.uint64))
    assert np.array_equal(got, np.array(want, dtype=np.uint32))


def test_device_philox_argument_checks():
    from paper_2202_00517_gb300 import _lib
    lib = _lib.load()
    assert lib.knnd_philox4x32_10(None, None, 0, None) == _lib.KNND_OK
    assert lib.knnd_philox4x32_10(None, None, 1, None) == _lib.KNND_EINVAL
    assert lib.knnd_philox4x32_10(None, None, -1, None) == _lib.KNND_EINVAL
