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
