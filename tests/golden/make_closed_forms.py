"""Writes sg_closed_forms.txt from the paper's closed forms (uses only `math`).

Per row: sharpness s, amplitude a (one channel), then
  max_v G  = a                       (Eq. 1 on the lobe axis, v = mu)
  min_v G  = a e^{-2 s}              (Eq. 1 at the antipode; Eq. 10's dynamic range is
                                      their difference, |a| (1 - e^{-2 s}))
  dc0      = a (1 - e^{-2 s}) / (2 s) (Eq. 12, the colour compensation)
"""
import math
import os

ROWS = [(0.5, 1.0), (1.0, 1.0), (1.0, -0.25), (3.7, 0.8), (12.0, 0.3), (50.0, -1.2)]

if __name__ == "__main__":
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "sg_closed_forms.txt")
    with open(out, "w") as f:
        f.write("# Spherical Gaussian closed forms, Eq. 1, Eq. 10 and Eq. 12 (Sec. 3.2, Sec. 3.3.3,\n")
        f.write("# Appendix derivation of the colour compensation). Written by make_closed_forms.py.\n")
        f.write("# s a G(v=mu) G(v=-mu) dc0\n")
        for s, a in ROWS:
            f.write(f"{s!r} {a!r} {a!r} {a * math.exp(-2 * s)!r} "
                    f"{a * (1 - math.exp(-2 * s)) / (2 * s)!r}\n")
    print(out)
