"""Philox4x64-10 counter-based generator and the noise maps built on it.

Oracle (test infrastructure only): imported by tests, ``__graft_entry__.smoke``
and the CPU-baseline leg of ``bench.py``; never by the product path.

The generator follows its published definition (Salmon, Moraes, Dror, Shaw,
"Parallel Random Numbers: As Easy as 1, 2, 3", SC'11): a 4x64-bit counter is
passed through 10 rounds of two 64x64->128 multiplies and an xor with the
key; the 2x64-bit key is bumped by two Weyl constants between rounds.

Noise vectors (Sec. 3, Eqs. iid_components1 / iid_components2):
  * Rademacher: x_i in {-1, +1}, equal probability.
  * Z4:         x_i in {1, i, -1, -i}, equal probability.
Bit mapping (the paper leaves it open; this is the project's definition):
  key     = (seed, (instance << 32) | (purpose << 8) | level)
  counter = (row_block, sample_index, 0, 0)
  Rademacher: row 256*row_block + 64*q + b takes bit b of output word q,
              0 -> +1, 1 -> -1.
  Z4:         row 128*row_block + 32*q + b takes bits (2b, 2b+1) of output
              word q as v in 0..3 (bit 2b least significant); x = i**v.
"""
import numpy as np

PHILOX_M0 = 0xD2E7470EE14C6C93
PHILOX_M1 = 0xCA5A826395121157
PHILOX_W0 = 0x9E3779B97F4A7C15
PHILOX_W1 = 0xBB67AE8584CAA73B
_MASK32 = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)

PURPOSE_NOISE = 0
PURPOSE_WARMUP = 1
PURPOSE_SETUP = 2


def _mulhilo(a, b):
    """(hi, lo) 64-bit halves of the 128-bit product of constant a and array b."""
    b = np.asarray(b, dtype=np.uint64)
    a = np.uint64(a)
    a0, a1 = a & _MASK32, a >> _S32
    b0, b1 = b & _MASK32, b >> _S32
    with np.errstate(over="ignore"):
        lo = a * b
        p00 = a0 * b0
        p01 = a0 * b1
        p10 = a1 * b0
        p11 = a1 * b1
        mid = p10 + (p00 >> _S32)
        mid2 = p01 + (mid & _MASK32)
        hi = p11 + (mid >> _S32) + (mid2 >> _S32)
    return hi, lo


def philox4x64_10(ctr, key):
    """Philox4x64 with 10 rounds.

    ctr: array (4, ...) of uint64; key: array (2, ...) of uint64 (broadcast).
    Returns an array (4, ...) of uint64.
    """
    c = [np.array(ctr[i], dtype=np.uint64) for i in range(4)]
    k0 = np.array(key[0], dtype=np.uint64)
    k1 = np.array(key[1], dtype=np.uint64)
    w0, w1 = np.uint64(PHILOX_W0), np.uint64(PHILOX_W1)
    for r in range(10):
        if r > 0:
            with np.errstate(over="ignore"):
                k0 = k0 + w0
                k1 = k1 + w1
        hi0, lo0 = _mulhilo(PHILOX_M0, c[0])
        hi1, lo1 = _mulhilo(PHILOX_M1, c[2])
        c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
    return np.stack(c)


def noise_key(seed, level, purpose=PURPOSE_NOISE, instance=0):
    return (np.uint64(seed), np.uint64((instance << 32) | (purpose << 8) | level))


def rademacher(n, seed, level, sample, purpose=PURPOSE_NOISE, instance=0):
    """Real noise vector of length n, entries +-1 (Eq. iid_components1)."""
    nblk = (n + 255) // 256
    k0, k1 = noise_key(seed, level, purpose, instance)
    blocks = np.arange(nblk, dtype=np.uint64)
    ctr = np.stack([blocks, np.full(nblk, sample, dtype=np.uint64),
                    np.zeros(nblk, np.uint64), np.zeros(nblk, np.uint64)])
    out = philox4x64_10(ctr, (k0, k1))          # (4, nblk)
    bits = (out.T[:, :, None] >> np.arange(64, dtype=np.uint64)) & np.uint64(1)
    bits = bits.reshape(nblk * 256)[:n]          # row = 256*blk + 64*q + b
    return 1.0 - 2.0 * bits.astype(np.float64)


def z4(n, seed, level, sample, purpose=PURPOSE_NOISE, instance=0):
    """Complex noise vector of length n, entries in {1, i, -1, -i} (Eq. iid_components2)."""
    nblk = (n + 127) // 128
    k0, k1 = noise_key(seed, level, purpose, instance)
    blocks = np.arange(nblk, dtype=np.uint64)
    ctr = np.stack([blocks, np.full(nblk, sample, dtype=np.uint64),
                    np.zeros(nblk, np.uint64), np.zeros(nblk, np.uint64)])
    out = philox4x64_10(ctr, (k0, k1))
    shifts = np.arange(0, 64, 2, dtype=np.uint64)
    v = (out.T[:, :, None] >> shifts) & np.uint64(3)
    v = v.reshape(nblk * 128)[:n].astype(np.int64)
    return np.array([1, 1j, -1, -1j], dtype=np.complex128)[v]


def noise(n, kind, seed, level, sample, purpose=PURPOSE_NOISE, instance=0):
    if kind == "rademacher":
        return rademacher(n, seed, level, sample, purpose, instance)
    if kind == "z4":
        return z4(n, seed, level, sample, purpose, instance)
    raise ValueError(kind)
