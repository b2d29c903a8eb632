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
