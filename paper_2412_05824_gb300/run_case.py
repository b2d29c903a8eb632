"""Run one plan configuration a few times on seeded inputs (for profiling a
single kernel under ncu).

    python -m paper_2412_05824_gb300.run_case DTYPE N FT DIRECTION REPS [LOG2_ELEMENTS [STRUCTURE]]

DTYPE float32|float64, FT off|detect|correct|correct_registers,
DIRECTION forward|inverse|inverse_unscaled; the batch is 2^LOG2_ELEMENTS / N
(default 2^26 elements); STRUCTURE default|split|cluster.
"""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))


def main(argv):
    import torch

    import paper_2412_05824_gb300 as tfl
    import synth_signals as ss

    dt, n, ft, d, reps = argv[0], int(argv[1]), argv[2], argv[3], int(argv[4])
    total = 1 << (int(argv[5]) if len(argv) > 5 else 26)
    x = ss.uniform_complex_torch(1, max(1, total // n), n, dt, device="cuda")
    y = torch.empty_like(x)
    structure = argv[6] if len(argv) > 6 else "default"
    p = tfl.Plan(n, x.shape[0], x.dtype, d, ft, structure=structure)
    for _ in range(reps):
        p.exec(x, y)
    torch.cuda.synchronize()
    print("ok", dt, n, ft, d, p.info())


if __name__ == "__main__":
    main(sys.argv[1:])
