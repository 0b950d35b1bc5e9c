"""Counter-based random numbers for the oracle (test infrastructure only).

The paper draws random numbers (commands, noise, pushes, curriculum loop-back, policy
sampling, minibatch shuffling) but fixes no generator.  Both the oracle and the CUDA path
implement, independently, one published counter-based construction so that the same
(seed, stream, counters, slot) gives the same 64-bit word on both sides:

* mixing function: the SplitMix64 output finaliser (Steele, Lea, Flood, "Fast splittable
  pseudorandom number generators", OOPSLA 2014; 64-bit constants of Vigna's public
  SplitMix64 reference implementation):
      z ^= z >> 30; z *= 0xBF58476D1CE4E5B9; z ^= z >> 27; z *= 0x94D049BB133111EB; z ^= z >> 31
* a key is built by chaining the finaliser over the counters, each added as (c + 1) * GAMMA
  with GAMMA = 0x9E3779B97F4A7C15 (the SplitMix64 increment);
* the slot-th word of a key is SplitMix64's slot-th output: mix64(key + (slot + 1) * GAMMA).

Derived variates (all integer / exactly representable, so both sides agree bit for bit):
* u32 = word >> 32; uniform01 = (u32 >> 8) * 2^-24 in [0, 1);
* uniform(-1, 1) = 2 * uniform01 - 1 (exact in fp32);
* mulhi32(u, n) = (u * n) >> 32, uniform on {0..n-1} (Lemire's multiply-shift);
* Irwin-Hall(4) normal (stand-in innovations): the four 16-bit fields of the word summed,
  centred, scaled by the fp32 constant 1/sqrt((2^32 - 1) / 3);
* Box-Muller normal (policy sampling, Sec. 2.2 Gaussian policy): u1 = ((hi >> 8) + 1) 2^-24 in
  (0, 1], u2 = (lo >> 8) 2^-24, eps = sqrt(-2 ln u1) cos(2 pi u2), evaluated in float64 here.

Pinned by tests/test_oracle_rng.py against the published SplitMix64 test vector (seed 0,
first outputs) and the moments of the derived variates.
"""
import numpy as np

MASK = (1 << 64) - 1
GAMMA = 0x9E3779B97F4A7C15
M1 = 0xBF58476D1CE4E5B9
M2 = 0x94D049BB133111EB

# Streams: one per consumer of randomness.
STREAM_ENV = 1
STREAM_ACT = 2
STREAM_PERM = 3
STREAM_INIT = 4
STREAM_TERRAIN = 5

# fp32 scale of the Irwin-Hall(4) normal: 1/sqrt((2^32-1)/3), stored as an exact fp32 value.
IH_SCALE = np.float32(float.fromhex("0x1.bb67aep-16"))


def mix64(z):
    """SplitMix64 finaliser on Python ints or numpy uint64 arrays (wrapping arithmetic)."""
    if isinstance(z, np.ndarray):
        z = z.astype(np.uint64)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(M1)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(M2)
        return z ^ (z >> np.uint64(31))
    z &= MASK
    z = ((z ^ (z >> 30)) * M1) & MASK
    z = ((z ^ (z >> 27)) * M2) & MASK
    return z ^ (z >> 31)


def _add_gamma(h, c):
    """h + (c + 1) * GAMMA mod 2^64 for int or uint64-array h and int or array counter c."""
    if isinstance(h, np.ndarray) or isinstance(c, np.ndarray):
        c = np.atleast_1d(np.asarray(c, dtype=np.uint64))
        h = np.atleast_1d(np.asarray(h, dtype=np.uint64))
        return h + (c + np.uint64(1)) * np.uint64(GAMMA)
    return (h + (c + 1) * GAMMA) & MASK


def key(seed, stream, a, b, env):
    """Per-(seed, stream, a, b, env) key: four chained finaliser rounds.

    (a, b) is (iteration, step) for the env and act streams, (iteration, epoch) for the
    permutation stream; env may be a numpy array of env ids.
    """
    h = mix64(_add_gamma(seed & MASK, stream))
    h = mix64(_add_gamma(h, a))
    h = mix64(_add_gamma(h, b))
    return mix64(_add_gamma(h, env))


def word(k, slot):
    """The slot-th 64-bit output of SplitMix64 started at key k."""
    return mix64(_add_gamma(k, slot))


def hi32(w):
    if isinstance(w, np.ndarray):
        return (w >> np.uint64(32)).astype(np.uint64)
    return w >> 32


def lo32(w):
    if isinstance(w, np.ndarray):
        return (w & np.uint64(0xFFFFFFFF)).astype(np.uint64)
    return w & 0xFFFFFFFF


def uniform01_f32(u32):
    """(u32 >> 8) * 2^-24 as float32 (exact)."""
    u = np.asarray(u32, dtype=np.uint64) >> np.uint64(8)
    return (u.astype(np.float32) * np.float32(2.0 ** -24)).astype(np.float32)


def uniform_pm1_f32(u32):
    """2 * uniform01 - 1 in float32 (both operations exact)."""
    return (np.float32(2.0) * uniform01_f32(u32) - np.float32(1.0)).astype(np.float32)


def mulhi32(u32, n):
    """floor(u32 * n / 2^32): uniform on {0, ..., n-1} (integer, exact)."""
    return ((np.asarray(u32, dtype=np.uint64) * np.uint64(n)) >> np.uint64(32)).astype(np.int64)


def irwin_hall_f32(w):
    """Approximately standard normal fp32 variate from one 64-bit word (exact on both sides).

    Sum of the four 16-bit fields (Irwin-Hall with n = 4), centred on its mean 131070, times
    IH_SCALE.  The centred sum is an integer of magnitude < 2^24, so its conversion to
    fp32 is exact and only the final product rounds.
    """
    w = np.asarray(w, dtype=np.uint64)
    s = np.zeros(w.shape, dtype=np.int64)
    for i in range(4):
        s += ((w >> np.uint64(16 * i)) & np.uint64(0xFFFF)).astype(np.int64)
    return ((s - 131070).astype(np.float32) * IH_SCALE).astype(np.float32)


def box_muller_f64(w):
    """Standard normal from one 64-bit word in float64 (cos branch of Box-Muller)."""
    w = np.asarray(w, dtype=np.uint64)
    u1 = ((hi32(w) >> np.uint64(8)).astype(np.float64) + 1.0) * 2.0 ** -24
    u2 = (lo32(w) >> np.uint64(8)).astype(np.float64) * 2.0 ** -24
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
