"""Philox4x32-10 and the sample-stream layout (oracle; test infrastructure).

Philox4x32-10 is the counter-based generator of Salmon, Moraes, Dror and Shaw
("Parallel random numbers: as easy as 1, 2, 3", SC'11).  The paper does not fix
a generator; the stream layout below is this project's convention and both the
oracle and the GPU implement it from this statement:

* counter = (sample_lo, sample_hi, iteration, (instance << 8) | block)
* key     = (seed_lo, seed_hi)
* block b of sample i yields words 4b .. 4b+3 of that sample's stream.
* a uniform is u = ((w >> 9) + 0.5) * 2**-23, which lies strictly inside (0, 1)
  and is exactly representable in FP32 and FP64.

Pinned against Triton's CPU-interpreted ``philox`` (a library routine) in
tests/test_oracle_philox.py.
"""
import numpy as np

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint64(0x9E3779B9)
_W1 = np.uint64(0xBB67AE85)
_MASK = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Ten Philox rounds on uint32 counters (arrays broadcast); returns 4 uint32 arrays."""
    c0 = np.asarray(c0, dtype=np.uint64) & _MASK
    c1 = np.asarray(c1, dtype=np.uint64) & _MASK
    c2 = np.asarray(c2, dtype=np.uint64) & _MASK
    c3 = np.asarray(c3, dtype=np.uint64) & _MASK
    k0 = np.asarray(k0, dtype=np.uint64) & _MASK
    k1 = np.asarray(k1, dtype=np.uint64) & _MASK
    for _ in range(10):
        p0 = _M0 * c0
        p1 = _M1 * c2
        hi0, lo0 = p0 >> _S32, p0 & _MASK
        hi1, lo1 = p1 >> _S32, p1 & _MASK
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0), lo1, (hi0 ^ c3 ^ k1), lo0
        k0 = (k0 + _W0) & _MASK
        k1 = (k1 + _W1) & _MASK
    return (c0.astype(np.uint32), c1.astype(np.uint32),
            c2.astype(np.uint32), c3.astype(np.uint32))


def stream_words(seed, iteration, instance, sample_index, n_words):
    """Words [n_words, N] of the stream of the given samples (sample_index: int array)."""
    i = np.asarray(sample_index, dtype=np.uint64)
    lo = i & _MASK
    hi = i >> _S32
    seed = int(seed)
    k0 = seed & 0xFFFFFFFF
    k1 = (seed >> 32) & 0xFFFFFFFF
    out = np.empty((n_words, i.size), dtype=np.uint32)
    for b in range((n_words + 3) // 4):
        c3 = ((int(instance) << 8) | b) & 0xFFFFFFFF
        r = philox4x32_10(lo, hi, int(iteration) & 0xFFFFFFFF, c3, k0, k1)
        for w in range(4):
            j = 4 * b + w
            if j < n_words:
                out[j] = r[w]
    return out


def words_to_uniform(w):
    """u = ((w >> 9) + 0.5) * 2**-23 in FP64 (exact)."""
    w = np.asarray(w, dtype=np.uint32)
    return ((w >> np.uint32(9)).astype(np.float64) + 0.5) * 2.0 ** -23


def uniforms(seed, iteration, instance, sample_index, dim):
    """Uniforms [dim, N] for the given samples."""
    return words_to_uniform(stream_words(seed, iteration, instance, sample_index, dim))
