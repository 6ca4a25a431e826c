"""Fit the odd polynomial used by the kernels' arctangent.

atan(a) for a in [0, 1] is approximated as a * P(a^2) with P of degree 7,
fitted by iteratively reweighted least squares on the relative error
(a Lawson-style minimax approximation), evaluated in FP64.  Prints the
coefficients (highest degree first, for Horner's scheme) and the maximum
absolute error; the kernel's table in brax_physics.cuh holds these values.

Usage: python paper_2106_13281_gb300/csrc/gen_atan_poly.py
"""
import numpy as np

DEG = 7


def fit(deg=DEG, n=20001, iters=60):
    a = np.cos(np.linspace(np.pi, 0, n)) * 0.5 + 0.5  # Chebyshev-spaced nodes on [0, 1]
    a = a[a > 0]
    s = a * a
    V = np.stack([s ** k for k in range(deg + 1)], axis=1) * a[:, None]
    y = np.arctan(a)
    w = np.ones_like(a)
    for _ in range(iters):
        c, *_ = np.linalg.lstsq(V * w[:, None], y * w, rcond=None)
        err = np.abs(V @ c - y)
        w = w * (err / err.max() + 1e-3)
        w /= w.max()
    return c


def main():
    c = fit()
    a = np.linspace(0, 1, 200001)
    approx = a * np.polyval(c[::-1], a * a)
    print("max abs error", np.abs(approx - np.arctan(a)).max())
    print("coefficients (s^7 ... s^0):")
    for v in c[::-1]:
        print(f"  {np.float32(v)!r}f,")
    # the same evaluation in FP32 Horner form
    cf = c[::-1].astype(np.float32)
    af = a.astype(np.float32)
    sf = af * af
    p = np.float32(0)
    for v in cf:
        p = p * sf + v
    print("FP32 max abs error", np.abs((af * p).astype(np.float64) - np.arctan(a)).max())


if __name__ == "__main__":
    main()
