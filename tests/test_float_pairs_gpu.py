"""Float-pair plans (TURBOFFT_STRUCTURE_FLOAT_PAIRS): complex128 transforms
computed in float-pair arithmetic instead of on the FP64 pipe, checked
element by element against the oracle at the float64 bar (relative L2 per
transform <= 5e-15 log2 N, maximum over transforms), in every direction,
on uniform and structured inputs, over one and two passes with ragged
batch tails."""
import numpy as np
import pytest

import oracle
import synth_signals as ss

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2412_05824_gb300 as tfl  # noqa: E402


def run(x, direction="forward"):
    batch, n = x.shape
    p = tfl.Plan(n, batch, "complex128", direction, "off", structure="float_pairs")
    y = p.exec(torch.from_numpy(np.ascontiguousarray(x)).cuda()).cpu().numpy()
    info = p.info()
    p.close()
    return y, info


def expected(x, direction):
    if direction == "forward":
        return oracle.fft(x)
    if direction == "forward_scaled":
        return oracle.fft(x) / x.shape[1]
    return oracle.fft(x, inverse=True, scaled=(direction == "inverse"))


def batch_for(n, target=1 << 18):
    b = max(1, target // n)
    return b + 3 if b > 4 else b


def check(x, direction="forward"):
    n = x.shape[1]
    y, info = run(x, direction)
    err = oracle.rel_l2(y, expected(x, direction))
    tol = oracle.tolerance(np.float64, n)
    assert np.all(np.isfinite(y))
    assert float(np.max(err)) <= tol, (n, direction, float(np.max(err)), tol)
    return float(np.max(err)) / tol, info


@pytest.mark.parametrize("n", [1 << k for k in range(3, 25)])
def test_forward_uniform(n):
    r, info = check(ss.uniform_complex(2, batch_for(n), n, np.float64))
    assert info["num_passes"] == (1 if n <= 4096 else 2)


@pytest.mark.parametrize("direction", ["inverse", "inverse_unscaled", "forward_scaled"])
@pytest.mark.parametrize("n", [8, 64, 512, 4096, 1 << 13, 1 << 16, 1 << 20])
def test_other_directions(direction, n):
    check(ss.uniform_complex(3, batch_for(n, 1 << 17), n, np.float64), direction)


@pytest.mark.parametrize("kind", ["impulse", "constant", "tone"])
@pytest.mark.parametrize("n", [8, 256, 4096, 1 << 14, 1 << 18])
def test_structured(kind, n):
    check(ss.structured(kind, 5, n, np.float64))


@pytest.mark.parametrize("scale", [2.0 ** -60, 2.0 ** -20, 2.0 ** 40, 2.0 ** 100])
def test_magnitudes_within_the_float_exponent_range(scale):
    # inputs of any magnitude inside the float range keep the relative bar
    x = ss.uniform_complex(4, 300, 1024, np.float64) * scale
    check(x)


def test_zeros_and_mixed_with_exact_zeros():
    x = ss.uniform_complex(5, 64, 512, np.float64)
    x[::3] = 0.0
    x[1::5, ::7] = 0.0
    y, _ = run(x)
    ref = oracle.fft(x)
    err = oracle.rel_l2(y, ref)
    assert np.all(y[::3] == 0)
    assert float(np.max(err)) <= oracle.tolerance(np.float64, 512)


def test_full_size_sampled():
    # the sweep's configuration: 2^28 elements, N = 2^12; a sample of
    # transforms checked against the oracle one by one
    n, batch = 4096, 1 << 16
    x = ss.uniform_complex_torch(2, batch, n, "float64", device="cuda")
    p = tfl.Plan(n, batch, "complex128", "forward", "off", structure="float_pairs")
    y = p.exec(x)
    idx = [0, 1, 777, batch // 2, batch - 2, batch - 1]
    xs = x[idx].cpu().numpy()
    err = oracle.rel_l2(y[idx].cpu().numpy(), oracle.fft(xs))
    assert float(np.max(err)) <= oracle.tolerance(np.float64, n)
    p.close()


@pytest.mark.parametrize("dtype,ft", [("complex64", "off"), ("complex128", "correct"), ("complex128", "detect")])
def test_unsupported(dtype, ft):
    with pytest.raises(tfl.TurboFFTError) as ei:
        tfl.Plan(1024, 4, dtype, "forward", ft, structure="float_pairs")
    assert ei.value.status == tfl.UNSUPPORTED
