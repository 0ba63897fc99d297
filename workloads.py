"""Seeded synthetic workloads of the differentially heated nanosuspension cavity.

Shared by the tests, the smoke check and the benchmark for both the CUDA path and the oracle.
It holds none of the method's arithmetic: only cavity sizes and parameters (the paper's
workloads restated as synthetic inputs: water / alumina, Sec. 2.d and Sec. 3) and seeded
random perturbations drawn with splitmix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), evaluated counter-style on (seed, field, node).
"""
import numpy as np

# 32 x 32, Ra 1e3, Pr 6.2, 1 % alumina of 20 nm in water, all slip forces, 2000 steps
CAVITY_32 = dict(name="cavity32_Ra1e3_phi1_dp20", nx=32, ny=32, Ra=1e3, Pr=6.2, phi=0.01,
                 d_p=20e-9, steps=2000)
# 256 x 256, Ra 1e5, 3 %, 30 nm, all slip forces, run towards steady state
CAVITY_256 = dict(name="cavity256_Ra1e5_phi3_dp30", nx=256, ny=256, Ra=1e5, Pr=6.2,
                  phi=0.03, d_p=30e-9, steps=200000)
# 1024 x 1024, Ra 1e6, 2 %, 50 nm: the state (226 MB in FP32) is larger than L2
CAVITY_1024 = dict(name="cavity1024_Ra1e6_phi2_dp50", nx=1024, ny=1024, Ra=1e6, Pr=6.2,
                   phi=0.02, d_p=50e-9, steps=0)

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(counter: np.ndarray) -> np.ndarray:
    """splitmix64 output for state = counter * golden gamma (uint64 in, uint64 out)."""
    with np.errstate(over="ignore"):
        z = (counter.astype(np.uint64) + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def uniform_pm1(seed: int, stream: int, n: int) -> np.ndarray:
    """n draws uniform in [-1, 1) for (seed, stream), float64 with 53 random bits."""
    idx = np.arange(n, dtype=np.uint64)
    base = np.uint64((int(seed) & 0xFFFFFF) << 40 | (int(stream) & 0xFF) << 32)
    u = (splitmix64(base + idx) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return 2.0 * u - 1.0


def perturbed_rest_fields(nx: int, ny: int, phi0: float, seed: int = 1, amp: float = 1e-3):
    """Initial (ux, uy, theta, phi) as float32 [4][ny][nx]: the fluid at rest, theta falling
    linearly from +1/2 at the hot wall to -1/2 at the cold wall, uniform phi0; plus seeded
    uniform noise of amplitude amp on ux, uy, theta and amp * phi0 on phi. float32 values
    are exactly representable on both sides, so both start from identical inputs."""
    n = nx * ny
    x = (np.arange(nx) + 0.5) / nx
    theta = np.broadcast_to(0.5 - x[None, :], (ny, nx))
    out = np.empty((4, ny, nx), dtype=np.float32)
    out[0] = (amp * uniform_pm1(seed, 0, n)).reshape(ny, nx)
    out[1] = (amp * uniform_pm1(seed, 1, n)).reshape(ny, nx)
    out[2] = theta + (amp * uniform_pm1(seed, 2, n)).reshape(ny, nx)
    out[3] = phi0 * (1.0 + amp * uniform_pm1(seed, 3, n)).reshape(ny, nx)
    return out


def random_state(nx: int, ny: int, seed: int, amp: float = 1.0) -> np.ndarray:
    """27 planes [27][ny][nx] of float32 uniform noise in [-amp, amp) (streaming tests)."""
    n = 27 * nx * ny
    return (amp * uniform_pm1(seed, 7, n)).astype(np.float32).reshape(27, ny, nx)


# Parametric sweep: Ra x phi x d_p, each cavity's resolution drawn from {64, 128, 256, 512}
# by splitmix64(seed 0, index) mod 4 (80 cavities).
SWEEP_RA = (1e3, 1e4, 1e5, 1e6)
SWEEP_PHI = (0.0, 0.01, 0.02, 0.03, 0.04)
SWEEP_DP = (10e-9, 30e-9, 50e-9, 100e-9)
SWEEP_SIZES = (64, 128, 256, 512)


def sweep80(seed: int = 0):
    """The 80 cavities of the sweep as dicts (nx, ny, Ra, Pr, phi, d_p), in a fixed order."""
    out = []
    idx = 0
    for Ra in SWEEP_RA:
        for phi in SWEEP_PHI:
            for d_p in SWEEP_DP:
                r = int(splitmix64(np.array([(int(seed) << 32) + idx], dtype=np.uint64))[0])
                n = SWEEP_SIZES[r % 4]
                out.append(dict(nx=n, ny=n, Ra=Ra, Pr=6.2, phi=phi, d_p=d_p))
                idx += 1
    return out


def random_net_params(segments, seed: int = 0, bias_scale: float = 0.05) -> np.ndarray:
    """Seeded network parameters (float32) for a list of (name, size, fan_in) segments: weights
    with fan_in > 0 uniform with the variance of He initialisation (2 / fan_in; 0.1 of that for
    the last conditioning layer "W2"), biases uniform in [-bias_scale, bias_scale]."""
    out = []
    for k, (name, size, fan_in) in enumerate(segments):
        u = uniform_pm1(seed, 200 + k, size)
        if fan_in > 0:
            a = np.sqrt(6.0 / fan_in) * (0.1 if name == "W2" else 1.0)
            out.append(a * u)
        else:
            out.append(bias_scale * u)
    return np.concatenate(out).astype(np.float32)


def random_conditions(n: int, seed: int) -> np.ndarray:
    """n cavity parameter points [n][3] (Ra, phi, d_p): log10 Ra uniform in [3, 6], phi uniform
    in [0, 0.05], d_p uniform in [10, 100] nm."""
    u = 0.5 * (uniform_pm1(seed, 7, 3 * n).reshape(n, 3) + 1.0)
    return np.stack([10.0 ** (3.0 + 3.0 * u[:, 0]), 0.05 * u[:, 1],
                     (10.0 + 90.0 * u[:, 2]) * 1e-9], axis=1)
