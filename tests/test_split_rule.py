"""Soundness of the split form's truncation rule, on the CPU.

The truncated split form drops the lowest weight diagonals of digit
products; what it drops sums to less than 2^ebits in units of the lowest
digit.  From the kept sum V it decides an output only when every value
within 2^ebits of V rounds to the same p-bit number: the round bit of |V|
lies at least two bits above ebits, and the bits between ebits and the
round bit are not all zero (round bit set: V is not on a midpoint's lower
edge) or all one (round bit clear: V is not just under a midpoint).
Otherwise the output goes to the exact kernel.

This restates that decision on Python integers and checks, against exact
round-to-nearest-even of the true sum, that no decided output can change
when the dropped part is added back -- on random sums and on sums placed at
the hard spots: just above and below midpoints and powers of two.
"""
import random

import pytest


def rn(x, p):
    """x rounded to p significant bits, nearest, ties to even (exact integers)."""
    a = abs(x)
    if a.bit_length() <= p:
        return x
    sh = a.bit_length() - p
    q, r = divmod(a, 1 << sh)
    half = 1 << (sh - 1)
    if r > half or (r == half and q & 1):
        q += 1
    return (q << sh) if x > 0 else -(q << sh)


def decided(v, p, ebits):
    """The truncation rule: True when the kept sum v alone fixes the rounding."""
    a = abs(v)
    if a == 0:
        return False
    lb = a.bit_length() - 1
    rb = lb - p
    if rb < ebits + 2:
        return False
    rbit = (a >> rb) & 1
    width = rb - ebits
    field = (a >> ebits) & ((1 << width) - 1)
    if rbit and field == 0:
        return False
    if not rbit and field == (1 << width) - 1:
        return False
    return True


def _hard_sums(rnd, p, ebits, count):
    """Sums near midpoints and powers of two, at random magnitudes."""
    out = []
    for _ in range(count):
        lb = p + ebits + rnd.randint(2, 40)
        q = (1 << (p - 1)) | rnd.getrandbits(p - 1)      # p significant bits
        base = q << (lb - p)                            # a p-bit number below 2^lb
        mid = base + (1 << (lb - p - 1))                # the midpoint above it
        pow2 = 1 << lb
        off = rnd.randint(-(1 << (ebits + 1)), 1 << (ebits + 1))
        for c in (base, mid, pow2):
            out.append(rnd.choice((1, -1)) * max(1, c + off))
    return out


@pytest.mark.parametrize("p", [53, 128, 512, 1024])
def test_decided_outputs_cannot_change(p):
    rnd = random.Random(p)
    decided_count = 0
    for ebits in (0, 5, 30, 77):
        sums = _hard_sums(rnd, p, ebits, 400)
        sums += [rnd.choice((1, -1)) * rnd.getrandbits(p + ebits + rnd.randint(0, 60)) for _ in range(400)]
        for v in sums:
            if not decided(v, p, ebits):
                continue
            decided_count += 1
            want = rn(v, p)
            lim = (1 << ebits) - 1
            for d in (-lim, lim, rnd.randint(-lim, lim), rnd.randint(-lim, lim)):
                assert rn(v + d, p) == want, (p, ebits, v, d)
    assert decided_count > 1000


def test_rule_defers_the_undecidable():
    """Exact midpoints, their near neighbours and small sums are left to the
    exact kernel."""
    p, ebits = 64, 10
    base = ((1 << (p - 1)) | 12345) << 41             # p significant bits, round bit at 40
    mid = base + (1 << 40)
    assert not decided(mid, p, ebits)                   # on a midpoint
    assert not decided(mid + 1, p, ebits)               # just above it: a dropped -2 would cross
    assert not decided(mid - 1, p, ebits)               # just below it
    assert decided(base + (1 << 39), p, ebits)          # a quarter ulp away: safe
    assert not decided(1 << (p + ebits), p, ebits)      # round bit too close to the dropped part
    assert not decided(0, p, ebits)
