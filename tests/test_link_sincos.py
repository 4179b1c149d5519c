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
    k = np.rint(th * K["kLinkInvPi"]).astype(f32)
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
    sign = np.where(k.astype(np.int64) % 2 == 1, f32(-1), f32(1))
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
