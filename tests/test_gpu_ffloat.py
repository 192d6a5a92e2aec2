"""The float-float sine and cosine of the time-marginalised kernel's per-sample set-up
against the FP64 sine and cosine of the library (torch on the device) and of numpy on the
host, and against what the mathematics fixes (sin^2 + cos^2 = 1; exact values at multiples
of pi/4; odd and even symmetry)."""
import math

import numpy as np
import pytest

from gpu_common import m, torch  # noqa: F401

pytestmark = pytest.mark.gpu


def _run(m, torch, x):
    xd = torch.tensor(x, dtype=torch.float64, device="cuda")
    s, c = torch.empty_like(xd), torch.empty_like(xd)
    m.mbis_debug_ff_sincos(len(x), xd, s, c)
    torch.cuda.synchronize()
    return xd, s, c


def test_ff_sincos_against_fp64(m, torch):
    rng = np.random.default_rng(20241005)
    near = np.concatenate([rng.uniform(-8 * np.pi, 8 * np.pi, 1 << 20),
                           (np.arange(-32, 33) * (np.pi / 4) + np.array([[-1e-7], [0.0], [1e-7]])).ravel(),
                           [0.0, -0.0, 5e-300, np.pi / 4, -np.pi / 4]])
    xd, s, c = _run(m, torch, near)
    es = (s - torch.sin(xd)).abs().max().item()
    ec = (c - torch.cos(xd)).abs().max().item()
    sh, ch = s.cpu().numpy(), c.cpu().numpy()
    print(f"  |x| < 8 pi: max |d sin| {es:.2e}, max |d cos| {ec:.2e} (device FP64)")
    assert es < 2e-13 and ec < 2e-13
    assert np.max(np.abs(sh - np.sin(near))) < 2e-13 and np.max(np.abs(ch - np.cos(near))) < 2e-13
    assert np.max(np.abs(sh * sh + ch * ch - 1.0)) < 5e-13
    # odd sine, even cosine on the same draws
    _, s2, c2 = _run(m, torch, -near)
    assert np.max(np.abs(s2.cpu().numpy() + sh)) < 2e-13 and np.max(np.abs(c2.cpu().numpy() - ch)) < 2e-13


def test_ff_sincos_exact_points_and_wide_angles(m, torch):
    k = np.arange(-16, 17)
    _, s, c = _run(m, torch, k * (np.pi / 2))
    np.testing.assert_allclose(s.cpu().numpy(), [(0, 1, 0, -1)[i % 4] for i in k], atol=1e-13)
    np.testing.assert_allclose(c.cpu().numpy(), [(1, 0, -1, 0)[i % 4] for i in k], atol=1e-13)
    _, s, c = _run(m, torch, np.array([math.pi / 6, math.pi / 3, 5 * math.pi / 6]))
    np.testing.assert_allclose(s.cpu().numpy(), [0.5, math.sqrt(3) / 2, 0.5], atol=1e-13)
    np.testing.assert_allclose(c.cpu().numpy(), [math.sqrt(3) / 2, 0.5, -math.sqrt(3) / 2], atol=1e-13)
    # wide angles: the reduction's FP64 pi/2 costs |k| 6e-17; past 2^20 the library's sincos
    wide = np.array([1e3, -7.5e4, 1e5 + 0.3, 1048575.9, 1048576.0, -3e7, 1e12])
    xd, s, c = _run(m, torch, wide)
    err = np.maximum(np.abs(s.cpu().numpy() - np.sin(wide)), np.abs(c.cpu().numpy() - np.cos(wide)))
    assert np.all(err <= np.maximum(2e-13, np.abs(wide) * 1e-16)), err
    m.mbis_debug_ff_sincos(0, None)
    with pytest.raises(m.MbisError):
        m.mbis_debug_ff_sincos(-1, xd)


def _basis(f):
    c = np.cbrt(f)
    return np.stack([1 / (f * c * c), 1 / f, 1 / (c * c), 1 / c, np.log(f), c, c * np.log(f), c * c, f])


@pytest.mark.parametrize("family", ["bns", "bbh"])
def test_float_float_set_up_against_fp64(m, torch, family):
    """The time-marginalised kernel's float-float per-sample set-up beside the FP64 one of
    the mixed kernels, on random parameters over each population's range: the phase they
    imply at every grid frequency agrees to 1e-9 turns, the amplitude to 1e-12 relative,
    the ISCO cut exactly."""
    rng = np.random.default_rng(2410 if family == "bns" else 5190)
    n = 20000
    if family == "bns":
        f_lo, df, nb = 20.0, 1.0 / 128, 128513
        p = [rng.uniform(0.9, 1.8, n), rng.uniform(1.0, 1.8, n), rng.uniform(-0.05, 0.05, n),
             rng.uniform(-0.05, 0.05, n), rng.uniform(-0.1, 0.1, n), rng.uniform(0, 2 * math.pi, n),
             rng.uniform(10, 400, n)]
    else:
        f_lo, df, nb = 20.0, 1.0 / 8, 8033
        p = [rng.uniform(8.0, 70.0, n), rng.uniform(1.0, 8.0, n), rng.uniform(-0.8, 0.8, n),
             rng.uniform(-0.8, 0.8, n), rng.uniform(-0.01, 0.01, n), rng.uniform(0, 2 * math.pi, n),
             rng.uniform(100, 3000, n)]
    params = torch.tensor(np.stack(p), dtype=torch.float64, device="cuda")
    out = torch.empty((24, n), dtype=torch.float64, device="cuda")
    m.mbis_debug_setup_pair(n, params, f_lo, df, nb, out)
    torch.cuda.synchronize()
    o = out.cpu().numpy()
    a, b = o[:12], o[12:]
    f = f_lo + df * np.array([0, 1, 10, 100, 1000, nb // 4, nb // 2, nb - 1], dtype=float)
    B = _basis(f)                                        # [9, n_f]
    dphase = (b[:9] - a[:9]).T @ B + (b[9] - a[9])[:, None]
    print(f"  {family}: max |d phase| {np.abs(dphase).max():.2e} turns, "
          f"max |d A / A| {np.max(np.abs(b[10] / a[10] - 1)):.2e}, cuts differing {int(np.sum(a[11] != b[11]))}")
    assert np.abs(dphase).max() <= 1e-9
    assert np.max(np.abs(b[10] / a[10] - 1)) <= 1e-12
    assert np.array_equal(a[11], b[11])
