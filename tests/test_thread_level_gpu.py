"""Thread-level ABFT (Sec. 4.2.1; mode TURBOFFT_FT_CORRECT_THREAD): where one
thread holds a whole transform, each thread checks its own transform with no
block reduction.  Parity with the oracle, no alarm on clean runs, injected
bit flips detected on the right transform and corrected back within the bar,
and the sizes it does not apply to rejected."""
import numpy as np
import pytest

import oracle
import synth_signals as ss

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2412_05824_gb300 as tfl  # noqa: E402

DT = {"complex64": np.float32, "complex128": np.float64}
CASES = [("complex64", 8, 3001), ("complex64", 16, 2003), ("complex64", 32, 1001),
         ("complex128", 8, 1501), ("complex128", 16, 777)]


@pytest.mark.parametrize("dtype,n,batch", CASES)
@pytest.mark.parametrize("direction", ["forward", "inverse"])
def test_parity_and_clean(dtype, n, batch, direction):
    x = ss.uniform_complex(21, batch, n, DT[dtype])
    ref = oracle.fft(x) if direction == "forward" else oracle.fft(x, inverse=True)
    p = tfl.Plan(n, batch, dtype, direction, "correct_thread")
    info = p.info()
    assert info["radix"][0] == n and info["num_passes"] == 1  # one thread per transform
    xd = torch.from_numpy(x).cuda()
    for _ in range(3):
        y = p.exec(xd).cpu().numpy()
        rep = p.report()
        assert rep["detected"] == 0 and rep["status"] == tfl.SUCCESS
        assert rep["groups_checked"] == batch  # every transform checked on its own
        assert 0 < rep["max_clean_ratio"] < 0.8
        assert float(np.max(oracle.rel_l2(y, ref))) <= oracle.tolerance(DT[dtype], n)
    p.close()


@pytest.mark.parametrize("dtype,n,batch", CASES)
def test_injected_faults_corrected(dtype, n, batch):
    x = ss.uniform_complex(22, batch, n, DT[dtype])
    ref = oracle.fft(x)
    tol = oracle.tolerance(DT[dtype], n)
    p = tfl.Plan(n, batch, dtype, "forward", "correct_thread")
    off = tfl.Plan(n, batch, dtype, "forward", "off")
    xd = torch.from_numpy(x).cuda()
    rng = np.random.default_rng(n * 7 + batch)
    exp_bit = 30 if dtype == "complex64" else 62
    man = list(range(10, 21)) if dtype == "complex64" else list(range(40, 51))
    detected = 0
    for k in range(16):
        tr, st, el, comp = int(rng.integers(0, batch)), int(rng.integers(0, 2)), int(rng.integers(0, n)), int(rng.integers(0, 2))
        bit = exp_bit if k % 2 == 0 else int(rng.choice(man))
        off.inject(tr, 0, st, el, comp, bit)
        e_off = oracle.rel_l2(off.exec(xd).cpu().numpy(), ref)
        p.inject(tr, 0, st, el, comp, bit)
        y = p.exec(xd).cpu().numpy()
        rep = p.report()
        if rep["detected"]:
            detected += 1
            assert rep["first_transform"] == tr and rep["corrected"] == 1 and rep["uncorrectable"] == 0, rep
        else:
            assert not (float(np.max(e_off)) > tol), (tr, st, el, comp, bit)  # no escape breaking the bar
        assert float(np.max(oracle.rel_l2(y, ref))) <= tol
    assert detected >= 8  # every exponent flip at least
    p.close()
    off.close()


def test_sizes_without_one_thread_shape_rejected():
    for dtype, n in (("complex64", 64), ("complex64", 1 << 16), ("complex128", 32), ("complex128", 4096)):
        with pytest.raises(tfl.TurboFFTError) as ei:
            tfl.Plan(n, 4, dtype, "forward", "correct_thread")
        assert ei.value.status == tfl.UNSUPPORTED
