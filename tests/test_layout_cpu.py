"""The AoSoA layout helpers of the inputs module (no GPU): component k of
track t of an array with K components per track sits at
((t // 32) * K + k) * 32 + t % 32."""
import numpy as np

from paper_2409_09228_gb300 import inputs


def test_aosoa_layout_round_trip():
    a = np.arange(3 * 2 * 70, dtype=np.float32).reshape(3, 2, 70)
    flat = inputs.to_aosoa32(a, 96)
    assert flat.shape == (3 * 2 * 96,)
    # component k of track t sits at ((t // 32) * K + k) * 32 + t % 32
    K = 6
    for k, t in ((0, 0), (5, 33), (3, 69)):
        assert flat[((t // 32) * K + k) * 32 + t % 32] == a.reshape(K, 70)[k, t]
    assert np.array_equal(inputs.from_aosoa32(flat, (3, 2, 96), 70), a)
