"""Richardson extrapolation and observed order (Sec. 3.3; oracle test utility).

For values f1, f2, f3 on meshes refined by a constant ratio c:
  extrapolated f = (f1 f3 - f2^2) / (f1 - 2 f2 + f3)
  observed order = ln((f2 - f1) / (f3 - f2)) / ln c
Pinned by the paper's printed example (Table rbc_richardson_values -> 0.52).
"""
import math


def extrapolate(f1, f2, f3):
    return (f1 * f3 - f2 * f2) / (f1 - 2.0 * f2 + f3)


def observed_order(f1, f2, f3, c):
    return math.log((f2 - f1) / (f3 - f2)) / math.log(c)
