"""The link-phase sine and cosine of the step kernel (link_sincos in
csrc/ahs_device.cuh), emulated step by step in float32 on the CPU: its constants
are the ones csrc/gen_link_sincos.py derives, and its error stays within the
bound its comment states (1.3e-7 for sin, 1.5e-7 for cos, about CUDA's 2-ulp
bound for sinf/cosf), against FP64 sin/cos of the same float32 angle.  The GPU
parity tests check the kernel that uses it against the oracle."""
import importlib.util
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2005_14454_gb300", "csrc")
f32 = np.float32


def constants():
    txt = open(os.path.join(CSRC, "ahs_device.cuh")).read()
    return {k: f32(float(v)) for k, v in re.findall(r"\b(kLink\w+)\s*=\s*([-+0-9.eE]+)f", txt)}


def fma(a, b, c):
    # float32 fused multiply-add: the product of two float32 values is exact in FP64
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(f32)


def link_sincos(th, K):
    th = th.astype(f32)
    full = lambda v: np.full(th.shape, v, f32)
    # k = rint(th / pi) from the rounding of t = 1.5 * 2^23 + th / pi (one FMA)
    t = fma(th, full(K["kLinkInvPi"]), full(K["kLinkRound"]))
    k = (t - K["kLinkRound"]).astype(f32)
    r = fma(-k, full(K["kLinkPiA"]), th)
    r = fma(-k, full(K["kLinkPiB"]), r)
    r2 = (r * r).astype(f32)
    ps = fma(r2, full(K["kLinkS3"]), full(K["kLinkS2"]))
    ps = fma(r2, ps, full(K["kLinkS1"]))
    ps = fma(r2, ps, full(K["kLinkS0"]))
    pc = fma(r2, full(K["kLinkC4"]), full(K["kLinkC3"]))
    pc = fma(r2, pc, full(K["kLinkC2"]))
    pc = fma(r2, pc, full(K["kLinkC1"]))
    pc = fma(r2, pc, full(K["kLinkC0"]))
    sv = fma((r * r2).astype(f32), ps, r)
    cv = fma(r2, pc, full(1.0))
    sign = np.where(t.view(np.uint32) & 1, f32(-1), f32(1))   # t's last bit: k's parity
    assert np.array_equal(t.view(np.uint32) & 1, k.astype(np.int64) & 1)
    return sv * sign, cv * sign


def test_constants_are_the_generators():
    spec = importlib.util.spec_from_file_location("gen", os.path.join(CSRC, "gen_link_sincos.py"))
    gen = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(gen)
    S, C, es, ec = gen.coefficients()
    K = constants()
    assert es < 1e-8 and ec < 1e-9
    for i, v in enumerate(S):
        assert K[f"kLinkS{i}"] == pytest.approx(v, rel=3e-7)
    for i, v in enumerate(C):
        assert K[f"kLinkC{i}"] == pytest.approx(v, rel=3e-7)
    assert K["kLinkPiA"] == f32(np.pi)
    assert K["kLinkPiB"] == f32(np.pi - float(f32(np.pi)))
    assert K["kLinkInvPi"] == f32(1 / np.pi)


@pytest.mark.parametrize("R", [4.0, 100.0, 1e4])
def test_error_bound(R):
    K = constants()
    th = np.random.default_rng(7).uniform(-R, R, 1_000_000).astype(f32)
    s, c = link_sincos(th, K)
    t = th.astype(np.float64)
    assert np.abs(s - np.sin(t)).max() <= 1.3e-7
    assert np.abs(c - np.cos(t)).max() <= 1.5e-7
    m2 = s.astype(np.float64) ** 2 + c.astype(np.float64) ** 2 - 1
    assert abs(m2.mean()) < 1e-8 and np.abs(m2).max() < 3e-7


def test_special_angles_and_symmetry():
    K = constants()
    th = np.array([0.0, np.pi / 2, np.pi, -np.pi, 1.5 * np.pi, 2 * np.pi, 1e-30, -1e-30, 3.0, -3.0], f32)
    s, c = link_sincos(th, K)
    assert s[0] == 0 and c[0] == 1
    assert np.allclose(s, np.sin(th.astype(np.float64)), atol=1.3e-7)
    assert np.allclose(c, np.cos(th.astype(np.float64)), atol=1.5e-7)
    # odd sine, even cosine, exactly (the reduction and polynomials are sign-symmetric)
    x = np.random.default_rng(1).uniform(-50, 50, 10000).astype(f32)
    s1, c1 = link_sincos(x, K)
    s2, c2 = link_sincos(-x, K)
    assert np.array_equal(s1, -s2) and np.array_equal(c1, c2)


def constants64():
    txt = open(os.path.join(CSRC, "ahs_device.cuh")).read()
    arr = {k: [float(v) for v in re.findall(r"[-+0-9.eE]+", body)]
           for k, body in re.findall(r"constexpr double (kLink[SC]64)\[8\] = \{([^}]*)\}", txt)}
    sc = {k: float(v) for k, v in re.findall(r"constexpr double (kLink\w+64) = ([-+0-9.eE]+);", txt)}
    return arr["kLinkS64"], arr["kLinkC64"], sc


def test_double_polynomials_fit_and_reduction():
    """FP64 link phases: the committed coefficients (exact arithmetic) are within
    1e-17 (sin, relative) and 5e-17 (cos) on [0, pi/2], and the whole evaluation in FP64 (reduction,
    polynomials, sign) within 3e-16 of the exact values for |th| up to 1e4."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    S, C, sc = constants64()
    assert len(S) == 8 and len(C) == 8
    assert sc["kLinkPiA64"] == np.pi and sc["kLinkInvPi64"] == 1 / np.pi
    assert sc["kLinkPiB64"] == float(mp.pi - mp.mpf(np.pi))
    worst_s = worst_c = 0.0
    for i in range(400):
        r = mp.mpf(i + 0.5) / 400 * mp.pi / 2
        r2 = r * r
        ps = sum(mp.mpf(S[j]) * r2 ** j for j in range(8))
        pc = sum(mp.mpf(C[j]) * r2 ** j for j in range(8))
        worst_s = max(worst_s, float(abs((r + r ** 3 * ps) - mp.sin(r)) / mp.sin(r)))
        worst_c = max(worst_c, float(abs((1 + r2 * pc) - mp.cos(r))))
    assert worst_s < 1e-17 and worst_c < 5e-17         # cos: the FP64 rounding of C0 ~ -1/2
    th = np.random.default_rng(9).uniform(-1e4, 1e4, 3000)
    # the fused multiply-adds of the reduction, each rounded once: k = rint(th / pi)
    # from t = 1.5 * 2^52 + th / pi, whose last bit is k's parity
    fma = lambda a, b_, c: float(mp.mpf(a) * mp.mpf(b_) + mp.mpf(c))
    t = np.array([fma(x, sc["kLinkInvPi64"], sc["kLinkRound64"]) for x in th])
    k = t - sc["kLinkRound64"]
    assert sc["kLinkRound64"] == 1.5 * 2.0 ** 52
    assert np.array_equal(t.view(np.int64) & 1, k.astype(np.int64) & 1)
    r = np.array([fma(-kk, sc["kLinkPiB64"], fma(-kk, sc["kLinkPiA64"], t)) for kk, t in zip(k, th)])
    r2 = r * r
    ps = np.full_like(r, S[7]); pc = np.full_like(r, C[7])
    for j in range(6, -1, -1):
        ps = r2 * ps + S[j]
        pc = r2 * pc + C[j]
    sgn = np.where(k.astype(np.int64) % 2 == 1, -1.0, 1.0)
    s, c = sgn * (r + r * r2 * ps), sgn * (1.0 + r2 * pc)
    es = max(abs(float(mp.mpf(a) - mp.sin(mp.mpf(t)))) for a, t in zip(s, th))
    ec = max(abs(float(mp.mpf(a) - mp.cos(mp.mpf(t)))) for a, t in zip(c, th))
    assert es < 3e-16 and ec < 3e-16, (es, ec)
