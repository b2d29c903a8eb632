"""The seeded input generators (shared by the oracle tests and the CUDA
parity tests): published SplitMix64 outputs, ranges, exact representability,
and agreement of the host (numpy) and torch implementations."""
import numpy as np
import torch

import synth_signals as ss


def test_splitmix64_published_stream():
    # SplitMix64 seeded with 1234567 (reference outputs of splitmix64.c)
    st = np.array([(1234567 + k * ss.GAMMA) & ss.MASK64 for k in range(1, 6)], dtype=np.uint64)
    got = [int(v) for v in ss._mix_np(st)]
    assert got == [6457827717110365317, 3203168211198807973, 9817491932198370423,
                   4593380528125082431, 16408922859458223821]


def test_uniform_range_and_precision():
    for dt in (np.float32, np.float64):
        x = ss.uniform_complex(1, 64, 1024, dt)
        assert x.dtype == (np.complex64 if dt == np.float32 else np.complex128)
        for part in (x.real, x.imag):
            assert part.min() >= -1.0 and part.max() < 1.0
            assert abs(part.mean()) < 0.01 and abs(part.var() - 1 / 3) < 0.01
    x32 = ss.uniform_complex(2, 4, 256, np.float32)
    # every value is a multiple of 2^-23 (exact in float32)
    k = (x32.real.astype(np.float64) + 1.0) * 2**23
    assert np.all(k == np.round(k))


def test_slices_match_full_batch():
    full = ss.uniform_complex(7, 10, 128, np.float32)
    part = ss.uniform_complex(7, 3, 128, np.float32, first_element=4 * 128)
    np.testing.assert_array_equal(full[4:7], part)


def test_torch_generator_bit_identical():
    for dt, name in ((np.float32, "float32"), (np.float64, "float64")):
        a = ss.uniform_complex(5, 3, 1000, dt)
        b = ss.uniform_complex_torch(5, 3, 1000, name, device="cpu").numpy()
        np.testing.assert_array_equal(a, b)


def test_structured_inputs():
    n = 48
    assert ss.tone_index(n) == 16 and ss.tone_index(1024) == 341
    t = ss.tone(2, 64, np.float64)
    np.testing.assert_allclose(np.abs(t), 1.0, atol=1e-15)
    assert ss.impulse(2, 8)[0, 0] == 1 and np.count_nonzero(ss.impulse(2, 8)) == 2
    assert np.all(ss.constant(1, 8) == 1)


def test_ragged_sizes_are_log_uniform_powers_of_two():
    s = ss.ragged_sizes(7, 22000, 6, 16)
    assert s.dtype == np.int64 and len(s) == 22000
    vals, counts = np.unique(s, return_counts=True)
    assert list(vals) == [1 << k for k in range(6, 17)]
    # 2000 expected per size; a 5-sigma band of the binomial
    assert np.all(np.abs(counts - 2000) < 5 * np.sqrt(2000))
    assert np.array_equal(s, ss.ragged_sizes(7, 22000, 6, 16))
    assert not np.array_equal(s, ss.ragged_sizes(8, 22000, 6, 16))
    # a prefix of a longer draw is the shorter draw (counter-based)
    assert np.array_equal(s[:100], ss.ragged_sizes(7, 100, 6, 16))


def test_ragged_offsets_pack_without_overlap():
    sizes = ss.ragged_sizes(3, 500, 3, 12)
    offs, total = ss.ragged_offsets(sizes)
    assert offs[0] == 0 and total == int(sizes.sum())
    assert np.array_equal(offs[1:], np.cumsum(sizes)[:-1])
    offs, total = ss.ragged_offsets(sizes, seed=9, max_gap=64)
    assert np.all(offs % 2 == 0)  # complex64 starts stay 16-byte aligned
    assert np.all(offs[1:] >= offs[:-1] + sizes[:-1])
    assert total == int(offs[-1] + sizes[-1]) and total >= int(sizes.sum())
    gaps = offs - np.concatenate([[0], offs[:-1] + sizes[:-1]])
    assert gaps.max() < 64 and gaps.max() > 0
