"""The octant argument behind the engine's winding count (csrc/ahs_device.cuh:
octant, winding): five angles in (-pi, pi] that add up to 2 pi W are each replaced
by the centre of their octant -- or of a neighbouring octant when they lie within
float32 rounding of its boundary -- and W = floor((2T + 9) / 16) of the summed
codes recovers W exactly.  Checked here on random plaquette-like angle sets,
including angles placed on octant boundaries; the GPU tests check the kernels'
windings against the oracle bit for bit."""
import numpy as np


def octant(a):
    return np.clip(np.floor(a * 4 / np.pi).astype(np.int64), -4, 3)


def wrap(a):
    return a + 2 * np.pi * np.floor((np.pi - a) / (2 * np.pi))


def test_octant_codes_recover_the_winding():
    rng = np.random.default_rng(3)
    n = 200_000
    # Y1 + Y2 - Y3 - Y4 + alpha = 2 pi W with alpha = [.]_pi of the remainder
    Y = rng.uniform(-np.pi, np.pi, (n, 4))
    Y[: n // 4] = np.round(Y[: n // 4] * 4 / np.pi) * np.pi / 4      # exactly on boundaries
    alpha = wrap(-(Y[:, 0] + Y[:, 1] - Y[:, 2] - Y[:, 3]))
    W = np.rint((Y[:, 0] + Y[:, 1] - Y[:, 2] - Y[:, 3] + alpha) / (2 * np.pi)).astype(np.int64)
    assert set(np.unique(W)) <= {-2, -1, 0, 1, 2} and (W != 0).any()
    angles = np.concatenate([Y, alpha[:, None]], axis=1)
    for trial in range(4):
        # rounding near a boundary may pick the neighbouring octant (never across +-pi)
        jitter = rng.uniform(-1e-6, 1e-6, angles.shape) * (trial > 0)
        o = octant(np.clip(angles + jitter, -np.pi + 1e-12, np.pi))
        T = o[:, 0] + o[:, 1] - o[:, 2] - o[:, 3] + o[:, 4]
        assert np.array_equal((2 * T + 9) >> 4, W)


def test_octant_of_complex_matches_the_angle():
    # the float32 classification by signs and |Re| vs |Im| against floor(4 arg / pi)
    rng = np.random.default_rng(4)
    a = rng.uniform(-np.pi, np.pi, 100_000)
    z = (np.cos(a) + 1j * np.sin(a)).astype(np.complex64)
    zr, zi = z.real, z.imag
    steep = np.abs(zi) > np.abs(zr)
    code = np.where(zi >= 0, np.where(zr >= 0, np.where(steep, 1, 0), np.where(steep, 2, 3)),
                    np.where(zr >= 0, np.where(steep, -2, -1), np.where(steep, -3, -4)))
    exact = octant(a)
    near = np.abs(a * 4 / np.pi - np.round(a * 4 / np.pi)) < 1e-5
    assert np.array_equal(code[~near], exact[~near])
    # at a boundary a neighbouring code; at +-pi the engine's near-cut fallback decides
    at_pi = np.abs(np.abs(a) - np.pi) < 1e-5
    assert (np.abs(code[near & ~at_pi] - exact[near & ~at_pi]) <= 1).all()


def flagged_code(zr, zi, tie):
    """The measuring kernel's flagged code (flagged_octant in csrc/ahs_device.cuh),
    restated: octant + 4 without branches -- 4 + 2b + (b xor s) for zi >= 0 and 7
    minus that below, b = (zr < 0), s = (|zi| > |zr|) -- and bit 3 when
    tie * zr + |zi| <= 0 (one fused multiply-add, emulated exactly in FP64)."""
    zr, zi = np.asarray(zr, np.float32), np.asarray(zi, np.float32)
    b = (zr < 0).astype(np.int64)
    s = (np.abs(zi) > np.abs(zr)).astype(np.int64)
    c = 4 + 2 * b + (b ^ s)
    c = np.where(zi < 0, 7 - c, c)
    near = (np.float32(tie).astype(np.float64) * zr.astype(np.float64) + np.abs(zi).astype(np.float64)
            ).astype(np.float32) <= 0
    return c | np.where(near, 8, 0)


def test_branch_free_code_is_the_octant():
    # every sign and steepness case, signed zeros included, and random values: the
    # branch-free code is octant + 4 of the select-based classification above
    vals = np.array([0.0, -0.0, 1.0, -1.0, 2.0, -2.0, 1e-30, -1e-30, 3.5, -3.5], np.float32)
    zr, zi = np.meshgrid(vals, vals)
    rng = np.random.default_rng(5)
    zr = np.concatenate([zr.ravel(), rng.uniform(-5, 5, 200_000).astype(np.float32)])
    zi = np.concatenate([zi.ravel(), rng.uniform(-5, 5, 200_000).astype(np.float32)])
    steep = np.abs(zi) > np.abs(zr)
    ref = np.where(zi >= 0, np.where(zr >= 0, np.where(steep, 1, 0), np.where(steep, 2, 3)),
                   np.where(zr >= 0, np.where(steep, -2, -1), np.where(steep, -3, -4))) + 4
    assert np.array_equal(flagged_code(zr, zi, 1e-5) & 7, ref)
    # away from the branch cut the angle's octant, and conjugation maps c to 7 - c
    a = rng.uniform(-np.pi, np.pi, 200_000)
    zr, zi = np.cos(a).astype(np.float32), np.sin(a).astype(np.float32)
    off = np.abs(a * 4 / np.pi - np.round(a * 4 / np.pi)) > 1e-5
    assert np.array_equal((flagged_code(zr, zi, 1e-5) & 7)[off], octant(a)[off] + 4)
    both = (zi != 0)
    assert np.array_equal((flagged_code(zr, -zi, 1e-5) & 7)[both], 7 - (flagged_code(zr, zi, 1e-5) & 7)[both])


def test_near_cut_flag_is_the_stated_window():
    # the flag marks zr <= 0 with |zi| <= tie |zr| (and z = 0); nothing with zr > 0
    # unless tie * zr underflows against zi = 0
    tie = 1e-5
    rng = np.random.default_rng(6)
    zr = rng.uniform(-2, 2, 400_000).astype(np.float32)
    zi = (rng.uniform(-2, 2, 400_000) * 10.0 ** rng.integers(-8, 1, 400_000)).astype(np.float32)
    flag = (flagged_code(zr, zi, tie) & 8) != 0
    window = (zr <= 0) & (np.abs(zi).astype(np.float64) <= tie * np.abs(zr).astype(np.float64))
    edge = np.abs(np.abs(zi).astype(np.float64) - tie * np.abs(zr).astype(np.float64)) <= 1e-7 * np.abs(zr)
    assert np.array_equal(flag[~edge], window[~edge]) and window.any() and (~window).any()
    assert (flagged_code(0.0, 0.0, tie) & 8) and (flagged_code(-0.0, -0.0, tie) & 8)
    assert not (flagged_code(1e-3, 0.0, tie) & 8) and not (flagged_code(-1.0, 1e-4, tie) & 8)
