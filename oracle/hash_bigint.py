"""Arbitrary-precision restatement of the seeded hash that picks S = Phi D.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Paper Section 2 defines the sparse embedding by a map h: [n] -> [t] and
independent signs D.  This build fixes a seeded 4-wise independent family:
two cubic polynomials over the prime field of p = 2^61 - 1 whose coefficients
come from the SplitMix64 stream started at ``seed`` (each 64-bit draw masked to
61 bits, the value p itself rejected); draws 0-3 are the bucket polynomial
c0..c3, draws 4-7 the sign polynomial.  For row index x:

    g(x) = c3*x**3 + c2*x**2 + c1*x + c0  (mod p)
    h(x) = g_bucket(x) mod m
    sigma(x) = +1 if g_sign(x) is even else -1

Python integers are exact, so this file evaluates the polynomial from its
definition (sum of powers), independently of the Horner / Mersenne-reduction
forms used elsewhere.
"""
from __future__ import annotations

P61 = (1 << 61) - 1
_MASK64 = (1 << 64) - 1


def splitmix64_stream(seed):
    """Generator of SplitMix64 outputs (Steele, Lea and Flood, OOPSLA 2014)."""
    state = seed & _MASK64
    while True:
        state = (state + 0x9E3779B97F4A7C15) & _MASK64
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        yield z ^ (z >> 31)


def coefficients(seed):
    """([c0..c3] of the bucket polynomial, [c0..c3] of the sign polynomial)."""
    out = []
    for z in splitmix64_stream(seed):
        c = z & P61
        if c == P61:
            continue
        out.append(c)
        if len(out) == 8:
            break
    return out[:4], out[4:]


def poly(c, x):
    return (c[3] * x ** 3 + c[2] * x ** 2 + c[1] * x + c[0]) % P61


def bucket_sign(seed, m, i):
    cb, cs = coefficients(seed)
    return poly(cb, i) % m, (1 if poly(cs, i) % 2 == 0 else -1)


def hash_rows(seed, m, rows):
    """Lists (buckets, signs) for an iterable of row indices."""
    cb, cs = coefficients(seed)
    hs, ss = [], []
    for i in rows:
        hs.append(poly(cb, i) % m)
        ss.append(1 if poly(cs, i) % 2 == 0 else -1)
    return hs, ss
