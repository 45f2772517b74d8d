"""Counter-based normals for Algorithm 1 step 4(a) ("generate xi ~ N(0, I)").

The paper only asks for i.i.d. standard normals.  The generator is fixed here so
that a GPU implementation written independently from the same published
definitions produces the same bits:

* Philox4x32-10, as defined by Salmon, Moraes, Dror and Shaw, "Parallel random
  numbers: as easy as 1, 2, 3" (SC'11): multipliers 0xD2511F53 / 0xCD9E8D57,
  Weyl key increments 0x9E3779B9 / 0xBB67AE85, ten rounds.
* key   = (seed mod 2^32, seed >> 32)
  counter = (q, sample mod 2^32, sample >> 32, level) for the q-th block of four
  normals, so normal j of a sample is word j mod 4 of block q = j div 4.
* uniforms: FP64  u = (x + 0.5) * 2^-32            (exact)
            FP32  u = (float(x) + 0.5f) * 2^-32    (float32 arithmetic)
* Box & Muller (1958): from (u0, u1) -> r cos(2 pi u1), r sin(2 pi u1) with
  r = sqrt(-2 ln u0); words (x0, x1) give normals 4q, 4q+1 and (x2, x3) give
  4q+2, 4q+3.
* ln, sin(pi t), cos(pi t) are evaluated with IEEE +, -, *, / and sqrt only, in
  a fixed order, so any IEEE-conforming implementation of the same steps is
  bit-identical:
    ln x: x = m 2^e with m in [sqrt(1/2), sqrt(2)); ln m = 2 atanh(f),
          f = (m-1)/(m+1), atanh(f)/f = sum_k f^(2k)/(2k+1) (the classical
          argument-reduction + atanh series, e.g. Cody & Waite 1980, ch. 5);
    sin/cos(pi t): t reduced by multiples of 1/2 (exact), then truncated
          Taylor series in x = pi r, |x| <= pi/4, in nested (Horner) form.
  Term counts: FP64 ln to s^10, sin to x^19, cos to x^18 (nested);
               FP32 ln to s^4,  sin to x^9,  cos to x^10 (Horner, with the
               coefficients rounded to float32 once; the next terms are
               below 2e-9, far under float32 resolution).
"""
import numpy as np

PHILOX_M0 = np.uint64(0xD2511F53)
PHILOX_M1 = np.uint64(0xCD9E8D57)
PHILOX_W0 = np.uint32(0x9E3779B9)
PHILOX_W1 = np.uint32(0xBB67AE85)
_MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32(counter, key, rounds=10):
    """Philox4x32-R block function on arrays of counters.

    counter: (4, N) uint32, key: (2,) or (2, N) uint32.  Returns (4, N) uint32.
    """
    c = [np.asarray(counter[i], dtype=np.uint32).copy() for i in range(4)]
    k0 = np.asarray(key[0], dtype=np.uint32).copy()
    k1 = np.asarray(key[1], dtype=np.uint32).copy()
    for r in range(rounds):
        if r > 0:
            k0 = ((k0.astype(np.uint64) + np.uint64(PHILOX_W0)) & _MASK32).astype(np.uint32)
            k1 = ((k1.astype(np.uint64) + np.uint64(PHILOX_W1)) & _MASK32).astype(np.uint32)
        p0 = PHILOX_M0 * c[0].astype(np.uint64)
        p1 = PHILOX_M1 * c[2].astype(np.uint64)
        hi0 = (p0 >> np.uint64(32)).astype(np.uint32)
        lo0 = (p0 & _MASK32).astype(np.uint32)
        hi1 = (p1 >> np.uint64(32)).astype(np.uint32)
        lo1 = (p1 & _MASK32).astype(np.uint32)
        c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
    return np.stack(c)


def philox_words(seed, level, sample, count):
    """The first `count` (multiple of 4) 32-bit words of one sample's stream."""
    assert count % 4 == 0
    q = np.arange(count // 4, dtype=np.uint64)
    assert count // 4 <= 2 ** 32
    ctr = np.stack([
        q.astype(np.uint32),
        np.full(q.shape, sample & 0xFFFFFFFF, dtype=np.uint32),
        np.full(q.shape, (sample >> 32) & 0xFFFFFFFF, dtype=np.uint32),
        np.full(q.shape, level & 0xFFFFFFFF, dtype=np.uint32),
    ])
    key = np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], dtype=np.uint32)
    out = philox4x32(ctr, key)          # (4, count/4)
    return out.T.reshape(-1)            # word j = out[j % 4, j // 4]


# ---------------------------------------------------------------- FP64 spec
_F64 = np.float64
_SQRT_HALF_64 = _F64(0.7071067811865476)
_LN2_64 = _F64(0.6931471805599453)
_PI_64 = _F64(3.141592653589793)


def log64(x):
    """ln x for x in (0, 1], FP64, by argument reduction + atanh series."""
    x = np.asarray(x, dtype=_F64)
    m, e = np.frexp(x)                      # exact: x = m * 2^e, m in [0.5, 1)
    e = e.astype(_F64)
    low = m < _SQRT_HALF_64
    m = np.where(low, m * _F64(2.0), m)     # exact
    e = np.where(low, e - _F64(1.0), e)
    f = (m - _F64(1.0)) / (m + _F64(1.0))
    s = f * f
    p = _F64(1.0) / _F64(21.0)
    for k in range(9, -1, -1):
        p = _F64(1.0) / _F64(2 * k + 1) + s * p
    t = f * p
    return e * _LN2_64 + (t + t)


def _reduce_half(t, dtype):
    """t = r + q/2 with integer q = rint(2t) and |r| <= 1/4 (exact)."""
    q = np.rint(t * dtype(2.0))
    r = t - q * dtype(0.5)
    return r, q.astype(np.int64) & 3


def sincospi64(t):
    """(sin(pi t), cos(pi t)) for t in [0, 2], FP64, Taylor series."""
    t = np.asarray(t, dtype=_F64)
    r, q = _reduce_half(t, _F64)
    x = _PI_64 * r
    x2 = x * x
    S = np.ones_like(x2)
    for k in range(9, 0, -1):
        S = _F64(1.0) - (x2 * S) * (_F64(1.0) / _F64((2 * k) * (2 * k + 1)))
    C = np.ones_like(x2)
    for k in range(9, 0, -1):
        C = _F64(1.0) - (x2 * C) * (_F64(1.0) / _F64((2 * k - 1) * (2 * k)))
    S = x * S
    sin = np.choose(q, [S, C, -S, -C])
    cos = np.choose(q, [C, -S, -C, S])
    return sin, cos


def normals64(seed, level, sample, count):
    """xi_j, j = 0..count-1, FP64 (count a multiple of 4)."""
    w = philox_words(seed, level, sample, count).reshape(-1, 4)
    u = (w.astype(_F64) + _F64(0.5)) * _F64(2.0 ** -32)
    out = np.empty((w.shape[0], 4), dtype=_F64)
    for a, b in ((0, 1), (2, 3)):
        r = np.sqrt(_F64(-2.0) * log64(u[:, a]))
        sn, cs = sincospi64(_F64(2.0) * u[:, b])
        out[:, a] = r * cs
        out[:, b] = r * sn
    return out.reshape(-1)


# ---------------------------------------------------------------- FP32 spec
_F32 = np.float32
_SQRT_HALF_32 = _F32(0.70710677)
_LN2_32 = _F32(0.6931472)
_PI_32 = _F32(3.1415927)
# (-1)^k / (2k+1)!, k = 0..4, and (-1)^k / (2k)!, k = 0..5, as float32
_SIN32 = [_F32(float.fromhex(h)) for h in
          ("0x1p0", "-0x1.555556p-3", "0x1.111112p-7", "-0x1.a01a02p-13", "0x1.71de3ap-19")]
_COS32 = [_F32(float.fromhex(h)) for h in
          ("0x1p0", "-0x1p-1", "0x1.555556p-5", "-0x1.6c16c2p-10", "0x1.a01a02p-16",
           "-0x1.27e4fcp-22")]


def log32(x):
    """ln x for x in (0, 1], float32 arithmetic throughout."""
    x = np.asarray(x, dtype=_F32)
    m, e = np.frexp(x)
    m = m.astype(_F32)
    e = e.astype(_F32)
    low = m < _SQRT_HALF_32
    m = np.where(low, m * _F32(2.0), m).astype(_F32)
    e = np.where(low, e - _F32(1.0), e).astype(_F32)
    f = (m - _F32(1.0)) / (m + _F32(1.0))
    s = f * f
    p = _F32(1.0) / _F32(9.0)
    for k in range(3, -1, -1):
        p = _F32(1.0) / _F32(2 * k + 1) + s * p
    t = f * p
    return (e * _LN2_32 + (t + t)).astype(_F32)


def sincospi32(t):
    """(sin(pi t), cos(pi t)) for t in [0, 2], float32 arithmetic."""
    t = np.asarray(t, dtype=_F32)
    r, q = _reduce_half(t, _F32)
    r = r.astype(_F32)
    x = _PI_32 * r
    x2 = x * x
    # Horner form, coefficients (-1)^k/(2k+1)! (sin, to x^9) and (-1)^k/(2k)!
    # (cos, to x^10) rounded to float32 once
    S = np.full_like(x2, _SIN32[-1])
    for c in _SIN32[-2::-1]:
        S = c + x2 * S
    C = np.full_like(x2, _COS32[-1])
    for c in _COS32[-2::-1]:
        C = c + x2 * C
    S = x * S
    sin = np.choose(q, [S, C, -S, -C]).astype(_F32)
    cos = np.choose(q, [C, -S, -C, S]).astype(_F32)
    return sin, cos


def normals32(seed, level, sample, count):
    """xi_j, j = 0..count-1, float32 spec (count a multiple of 4)."""
    w = philox_words(seed, level, sample, count).reshape(-1, 4)
    u = (w.astype(_F32) + _F32(0.5)) * _F32(2.0 ** -32)
    out = np.empty((w.shape[0], 4), dtype=_F32)
    for a, b in ((0, 1), (2, 3)):
        r = np.sqrt(_F32(-2.0) * log32(u[:, a]))
        sn, cs = sincospi32(_F32(2.0) * u[:, b])
        out[:, a] = r * cs
        out[:, b] = r * sn
    return out.reshape(-1)


def normals(seed, level, sample, count, precision=64):
    return normals64(seed, level, sample, count) if precision == 64 else \
        normals32(seed, level, sample, count)
