"""Write tf_dft_constants.h: cos and sin of 2*pi*q/32, q = 0..31, to 20
significant digits (evaluated with mpmath at 40 digits), as constexpr
functions so that butterfly twiddles fold into immediates.  These are the
constant twiddles of the register-level radix-2..32 butterflies."""
import os

import mpmath as mp

mp.mp.dps = 40
HERE = os.path.dirname(os.path.abspath(__file__))


def _fmt(v):
    s = mp.nstr(v, 21, min_fixed=-30, max_fixed=30)
    return s if ("." in s or "e" in s) else s + ".0"


def main():
    lines = [
        "// Generated by gen_dft_constants.py: cos/sin(2*pi*q/32), q = 0..31.",
        "#pragma once",
        "namespace tf {",
        "__host__ __device__ constexpr double cos32(int q) {",
        "  switch (q & 31) {",
    ]
    for q in range(32):
        lines.append("    case %d: return %s;" % (q, _fmt(mp.cos(2 * mp.pi * q / 32))))
    lines += ["  }", "  return 0.0;", "}", "__host__ __device__ constexpr double sin32(int q) {", "  switch (q & 31) {"]
    for q in range(32):
        lines.append("    case %d: return %s;" % (q, _fmt(mp.sin(2 * mp.pi * q / 32))))
    lines += ["  }", "  return 0.0;", "}", "}  // namespace tf", ""]
    with open(os.path.join(HERE, "tf_dft_constants.h"), "w") as f:
        f.write("\n".join(lines))


if __name__ == "__main__":
    main()
