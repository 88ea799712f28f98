"""The split products' digit extraction in closed form.

The FP64-accurate products cut every scaled operand value, held as a 64-bit
integer y with |y| <= 2^62, into signed 7-bit digits by sequential rounding:
digit k is y_(k-1) / 2^d_k rounded half up, d_k = 62 - 7k, and y_k the
remainder.  The kernel computes the same digits in closed form: with R_k the
rounding of y itself to a multiple of 2^d_k, the first k digits sum to
R_k 2^d_k, so q_1 = R_1 and q_k = R_k - 2^7 R_(k-1), and only the low 32 bits
of each R_k are needed because every q_k is small.  This checks the identity,
the digit bounds and the remainder bound in exact integer arithmetic, with
the 32-bit wrap-around the kernel relies on, including ties."""
import random

SPLIT_BITS = 7


def sequential(y, ns):
    q = []
    for k in range(1, ns + 1):
        d = 62 - SPLIT_BITS * k
        qk = (y + (1 << (d - 1))) >> d
        y -= qk << d
        q.append(qk)
    return q, y


def closed_form_32bit(y, ns):
    q, rprev = [], 0
    for k in range(1, ns + 1):
        d = 62 - SPLIT_BITS * k
        t = (y + (1 << (d - 1))) & ((1 << 64) - 1)  # unsigned 64-bit add
        lo, hi = t & 0xFFFFFFFF, t >> 32
        if d >= 32:
            r = (hi - (1 << 32) if hi >= 1 << 31 else hi) >> (d - 32)  # arithmetic shift of the signed high word
        else:
            r = (((hi << 32) | lo) >> d) & 0xFFFFFFFF  # funnel shift: low 32 bits
            r = r - (1 << 32) if r >= 1 << 31 else r
        if k == 1:
            qk = r
        else:
            qk = (r - (rprev << 7)) & 0xFFFFFFFF
            qk = qk - (1 << 32) if qk >= 1 << 31 else qk
        q.append(qk)
        rprev = r
    return q


def cases(rng):
    for _ in range(20000):
        yield rng.randint(-(1 << 62), 1 << 62)
    for k in range(1, 9):
        d = 62 - SPLIT_BITS * k
        for m in range(-300, 301):
            for dd in (-1, 0, 1):
                y = m * (1 << (d - 1)) + dd
                if abs(y) <= 1 << 62:
                    yield y


def test_closed_form_equals_sequential_rounding():
    rng = random.Random(5)
    for y in cases(rng):
        for ns in range(3, 9):
            q, rem = sequential(y, ns)
            assert closed_form_32bit(y, ns) == q, (y, ns)
            # bounds the split products' error analysis rests on
            assert abs(q[0]) <= 128 and all(abs(x) <= 64 for x in q[1:])
            d = 62 - SPLIT_BITS * ns
            assert -(1 << (d - 1)) <= rem < (1 << (d - 1))
            assert sum(x << (62 - SPLIT_BITS * (k + 1)) for k, x in enumerate(q)) + rem == y


def test_digits_do_not_depend_on_the_slice_count():
    """Slices computed for s serve any product with fewer: digit k is the same
    for every slice count that includes it."""
    rng = random.Random(6)
    for _ in range(5000):
        y = rng.randint(-(1 << 62), 1 << 62)
        full = closed_form_32bit(y, 8)
        for ns in range(3, 8):
            assert closed_form_32bit(y, ns) == full[:ns]
