"""Accuracy of the kernels' arctangent (GPU).

The joint limits (App. A angle_limit) measure hinge angles with the
kernels' own four-quadrant arctangent: an octant reduction and a degree-7
odd polynomial fitted for this library, at most 1.3e-7 rad off atan on
[0, 1] when evaluated in FP32.  Here it runs elementwise through the
library's probe entry point over every octant and many magnitudes, and is
compared with FP64 atan2 of the same FP32 inputs and with CUDA's atan2f
(torch.atan2 on the device)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def probe(y, x):
    from paper_2106_13281_gb300.binding import _ptr, _stream, check, load_library
    L = load_library()
    yd, xd = torch.from_numpy(y).cuda(), torch.from_numpy(x).cuda()
    out, outp = torch.empty_like(yd), torch.empty_like(yd)
    check(L.brax_internal_atan2(_ptr(yd), _ptr(xd), _ptr(out), _ptr(outp), y.size, _stream()))
    torch.cuda.synchronize()
    return out.cpu().numpy(), outp.cpu().numpy(), torch.atan2(yd, xd).cpu().numpy()


def test_fast_atan2_error_bound_all_octants():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    rng = np.random.default_rng(0)
    n = 1 << 20
    ang = rng.uniform(-np.pi, np.pi, n)
    mag = 10.0 ** rng.uniform(-6, 6, n)
    y = (mag * np.sin(ang)).astype(np.float32)
    x = (mag * np.cos(ang)).astype(np.float32)
    # octant boundaries, axes and the origin
    sp = np.array([[0, 1], [1, 1], [1, 0], [1, -1], [0, -1], [-1, -1], [-1, 0], [-1, 1], [0, 0],
                   [1e-30, 1], [1, 1e-30], [-1e-30, -1], [3, 3 + 1e-6]], dtype=np.float32)
    y = np.concatenate([y, sp[:, 0]])
    x = np.concatenate([x, sp[:, 1]])
    got, got_packed, cuda_atan2 = probe(y, x)
    ref = np.arctan2(y.astype(np.float64), x.astype(np.float64))
    # the fit's 1.3e-7 rad plus the FP32 rounding of the octant steps
    # (pi/2 - r, pi - r): one unit in the last place of the result
    bound = 1.3e-7 + np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64)
    err = np.abs(got.astype(np.float64) - ref)
    assert (err <= bound).all(), float((err - bound).max())
    assert np.abs(err).max() < 3.7e-7
    first = (x > 0) & (np.abs(y) <= x) & (np.abs(ref) < 0.5)
    assert np.abs(err[first]).max() <= 1.3e-7 + 6e-8
    # CUDA's atan2f (within 2 ulp of the exact value) agrees within both bounds
    assert (np.abs(got.astype(np.float64) - cuda_atan2.astype(np.float64)) <= bound + 2 * np.spacing(
        np.abs(cuda_atan2))).all()
    assert got[-5] == 0.0  # atan2(0, 0)
    # the packed two-environment form computes the same FP32 operations
    assert np.array_equal(got, got_packed)
