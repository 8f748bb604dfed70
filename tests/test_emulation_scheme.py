"""The arithmetic of the emulated FP64 product (FP64 path 2), checked in exact
integer and rational arithmetic on the CPU: the slicing of a double into eight
balanced base-128 digits under its row's power of two, the exactness budget of
the fp32 group sums, and the error of the whole scheme against the exact
product.  These pin the claims the CUDA kernel is built on; the kernel itself is
checked against an extended-precision reference by the GPU tests."""
from fractions import Fraction

import numpy as np

S, BETA, KC = 8, 7, 512


def expo_field(v):
    u = np.float64(v).view(np.uint64)
    e = int((u >> np.uint64(52)) & np.uint64(0x7FF))
    return 1 if (e == 0 and v != 0) else e


def scaled_int(v, E):
    """X = round(v 2^(1078 - E)) (half up on the magnitude), from the bit pattern."""
    u = int(np.float64(v).view(np.uint64))
    f = (u >> 52) & 0x7FF
    m = u & ((1 << 52) - 1)
    if f == 0:
        f = 1
    else:
        m |= 1 << 52
    sh = f - E + 3
    if sh >= 0:
        a = m << sh
    elif sh <= -63:
        a = 0
    else:
        a = (m + (1 << (-sh - 1))) >> (-sh)
    return -a if u >> 63 else a


def digits(v, E):
    """Balanced base-128 digits of X = round(v 2^(1078 - E)), most significant first."""
    X = scaled_int(v, E)
    t = [0] * S
    for i in range(S - 1, 0, -1):
        d = X & 127
        d = d - 128 if d >= 64 else d
        t[i] = d
        X = (X - d) >> 7
    t[0] = X
    return t


def test_digits_reconstruct_the_scaled_value():
    rng = np.random.default_rng(0)
    vals = np.concatenate([rng.standard_normal(300) * 10.0 ** rng.uniform(-8, 8, 300), [0.0, -0.0, 1.0, -1.0]])
    E = max(expo_field(v) for v in vals)
    scale = Fraction(2) ** (E - 1022)
    for v in vals:
        t = digits(v, E)
        assert abs(t[0]) <= 128 and all(-64 <= d <= 63 for d in t[1:])
        rec = scale * sum(Fraction(d) * Fraction(2) ** (-BETA * (i + 1)) for i, d in enumerate(t))
        # rounding to 57 fractional bits of the row scale: |v - rec| <= 2^-57 scale
        assert abs(Fraction(float(v)) - rec) <= scale * Fraction(1, 2 ** 57)
        # every digit is exact in bf16 (at most 8 significant bits)
        for d in t:
            f = np.float32(d)
            assert (f.view(np.uint32) & 0xFFFF) == 0


def test_rows_of_subnormals_keep_their_values():
    """A subnormal entry's exponent field counts as 1 (the scale of the smallest normal), so a
    row whose largest entry is subnormal is sliced exactly, not dropped as a zero row."""
    tiny = 2.0 ** -1074
    for row in ([tiny, -3 * tiny, 1e-310, -2.2e-308], [1e-310, 0.0, -0.0], [2.0 ** -1022, 1e-315]):
        E = max(expo_field(v) for v in row)
        assert E == 1
        scale = Fraction(2) ** (E - 1022)
        for v in row:
            t = digits(v, E)
            rec = scale * sum(Fraction(d) * Fraction(2) ** (-BETA * (i + 1)) for i, d in enumerate(t))
            assert rec == Fraction(float(v))                 # exact: subnormals are multiples of 2^-1074
            assert digits_offset_form(v, E) == t


def digits_offset_form(v, E):
    """The kernels' form of the same digits: Y = X + sum_{j<7} 64 2^(7 j); the low seven
    digits are the base-128 digits of Y less 64, the top digit is Y >> 49 (arithmetic),
    and each low digit reaches bf16 as the float 2^23 + u less 2^23 + 64 (u = digit + 64)."""
    Y = scaled_int(v, E) + sum(64 << (7 * j) for j in range(7))
    t = [Y >> 49] + [((Y >> (7 * (S - 1 - i))) & 127) - 64 for i in range(1, S)]
    for i in range(1, S):
        u = t[i] + 64
        f = np.float32(np.uint32(0x4B000000 | u).view(np.float32)) - np.float32(8388672.0)
        assert f == np.float32(t[i])
    return t


def test_offset_form_gives_the_same_digits():
    rng = np.random.default_rng(4)
    vals = np.concatenate([rng.standard_normal(2000) * 10.0 ** rng.uniform(-12, 12, 2000),
                           [0.0, -0.0, 1.0, -1.0, 2.0 ** -60, -(2.0 ** 30)]])
    for E in (max(expo_field(v) for v in vals), 1023, 1050):
        for v in vals:
            if expo_field(v) <= E:
                assert digits_offset_form(v, E) == digits(v, E)


def test_group_sums_within_fp32_exact_range():
    """Worst case over K = 512 terms: group G collects the products (i, G - i);
    the groups G <= 5 stay within 2^24 (exact in fp32), the two lowest may round."""
    top = {}
    for G in range(8):
        members = [(i, G - i) for i in range(G + 1) if G - i < S]
        per_term = sum((128 if i == 0 else 64) * (128 if j == 0 else 64) for i, j in members)
        top[G] = KC * per_term
    assert all(top[G] <= 2 ** 24 for G in range(6))
    assert top[6] > 2 ** 24 and top[7] < 2 ** 31        # still exact as integers after conversion
    # their rounding is at most K ulps of 2 at weights 2^-56 and 2^-63 of the output scale
    assert KC * 2 * 2.0 ** (-7 * 8) <= 2.0 ** -46


def scheme_product(A, B):
    """The emulated product op(A) op(B) in exact integer arithmetic, as the kernels
    compute it for one K chunk (K <= 512): digits under each row's and column's
    power of two, the 36 slice products of groups G = i + j <= 7 summed per group,
    each group sum through an fp32 accumulator, the groups combined exactly and
    rounded once to a double."""
    m, k = A.shape
    n = B.shape[1]
    Ea = [max(expo_field(v) for v in A[r]) for r in range(m)]
    Eb = [max(expo_field(v) for v in B[:, c]) for c in range(n)]
    ta = [[digits(A[r, q], Ea[r]) for q in range(k)] for r in range(m)]
    tb = [[digits(B[q, c], Eb[c]) for q in range(k)] for c in range(n)]
    C = np.zeros((m, n))
    for r in range(m):
        for c in range(n):
            acc = [sum(ta[r][q][i] * tb[c][q][G - i] for q in range(k) for i in range(G + 1)) for G in range(8)]
            acc = [int(np.float32(a)) for a in acc]                  # the fp32 accumulators
            hi = ((acc[0] * 128 + acc[1]) * 128 + acc[2]) * 128 + acc[3]
            lo = ((acc[4] * 128 + acc[5]) * 128 + acc[6]) * 128 + acc[7]
            t = float(Fraction(hi) * 2 ** 28 + lo)                   # one rounding
            C[r, c] = t * 2.0 ** (Ea[r] + Eb[c] - 2107)
    return C


def _exact_product(A, B):
    return [[sum(Fraction(float(A[r, q])) * Fraction(float(B[q, c])) for q in range(A.shape[1]))
             for c in range(B.shape[1])] for r in range(A.shape[0])]


def normwise_bound(A, B, exact):
    """|C_ij - (AB)_ij| <= u |(AB)_ij| + K 2^-52 max_k |A_ik| max_k |B_kj| (one K chunk)."""
    k = A.shape[1]
    ra = np.abs(A).max(axis=1)
    cb = np.abs(B).max(axis=0)
    return [[Fraction(2.0 ** -53) * abs(exact[r][c]) + Fraction(k * 2.0 ** -52 * float(ra[r] * cb[c]))
             for c in range(B.shape[1])] for r in range(A.shape[0])]


def test_scheme_error_against_exact_product():
    rng = np.random.default_rng(1)
    m, n, k = 6, 5, 40
    A = rng.standard_normal((m, k)) * 10.0 ** rng.uniform(-4, 4, (m, 1))
    B = rng.standard_normal((k, n)) * 10.0 ** rng.uniform(-4, 4, (1, n))
    A[0, 3] *= 1e-12
    C = scheme_product(A, B)
    exact = _exact_product(A, B)
    bound = normwise_bound(A, B, exact)
    for r in range(m):
        for c in range(n):
            assert abs(Fraction(C[r, c]) - exact[r][c]) <= bound[r][c], (r, c)


def test_uneven_row_exceeds_the_elementwise_bound_and_meets_the_normwise_one():
    """a = [1, 1.23e-9] against b = [0, 1]: the exact product is the small entry
    alone, which the row's scale keeps to 2^-57 of 1 only.  The error is far above
    the elementwise bound 4 u |a||b| of an FP64 dot product and within the normwise
    bound of the scheme."""
    A = np.array([[1.0, 1.23e-9]])
    B = np.array([[0.0], [1.0]])
    C = scheme_product(A, B)
    exact = _exact_product(A, B)
    err = abs(Fraction(C[0, 0]) - exact[0][0])
    assert err > 1e6 * Fraction(4 * 2.0 ** -53 * 1.23e-9)
    assert err <= normwise_bound(A, B, exact)[0][0]


def test_normwise_bound_on_adversarial_operands():
    """Rows with one entry of order one and the rest spread over 1e-3 .. 1e-15,
    columns that zero or keep the large entry, K up to 512 (one chunk, where the
    fp32 group sums of G = 6 can exceed 2^24 and round): the bound holds and is
    within a modest factor of the error for the worst element."""
    rng = np.random.default_rng(6)
    worst = 0.0
    for k in (3, 64, 512):
        m, n = 3, 3
        A = rng.standard_normal((m, k)) * 10.0 ** rng.uniform(-15, -3, (m, k))
        A[:, 0] = rng.uniform(1.0, 2.0, m)
        B = rng.standard_normal((k, n)) * 10.0 ** rng.uniform(-15, 0, (k, n))
        B[0, 0] = 0.0
        if k == 512:                     # all-maximal digits: the fp32 group sums round
            A[1] = 2.0 - 2.0 ** -52
            B[:, 2] = -(2.0 - 2.0 ** -52)
        C = scheme_product(A, B)
        exact = _exact_product(A, B)
        bound = normwise_bound(A, B, exact)
        for r in range(m):
            for c in range(n):
                err = abs(Fraction(C[r, c]) - exact[r][c])
                assert err <= bound[r][c], (k, r, c)
                worst = max(worst, float(err / bound[r][c]))
    assert worst > 1e-3


def _to_double(hi, lo, e, neg):
    """The combination's rounding of V = hi 2^28 + lo (|hi|, |lo| < 2^47) to a double
    times 2^e, transcribing the CUDA kernel's straight-line integer arithmetic: V = H 2^28 + L
    with 0 <= L < 2^28, |V| as (Hm, Lm); both justifications of the 64-bit word N and the
    case Hm = 0 computed with shift amounts kept in range, then selected; N rounded at its
    bit 11; the biased exponent added onto the rounded significand; infinity above the
    normal range, the subnormal grid (q rounded once more) below it.  Returns the double and
    the rounded significand q and leading-bit index P."""
    import struct
    m64, m32 = (1 << 64) - 1, (1 << 32) - 1
    clz64 = lambda x: 64 - x.bit_length()
    clz32 = lambda x: 32 - x.bit_length()
    H, L = hi + (lo >> 28), lo & 0xFFFFFFF
    assert H * 2 ** 28 + L == hi * 2 ** 28 + lo and 0 <= L < 2 ** 28
    sv = H < 0
    Hm = (((~H) if L else -H) if sv else H) & m64
    Lm = ((0x10000000 - L) & 0xFFFFFFF) if sv else L
    assert Hm * 2 ** 28 + Lm == abs(H * 2 ** 28 + L)
    lzh = clz64(Hm) & 63
    right = lzh < 28
    low = (Lm >> (28 - lzh if right else 0)) if right else ((Lm << (0 if right else lzh - 28)) & m64)
    NH = ((Hm << lzh) & m64) | low
    stH = ((Lm << ((lzh + 4) & 31)) & m32) if right else 0
    lzl = clz32(Lm)
    NL = (Lm << ((lzl + 32) & 63)) & m64
    hz = Hm == 0
    N = NL if hz else NH
    sticky = 0 if hz else stH
    P = 31 - lzl if hz else 91 - lzh
    if (Hm | Lm) == 0:
        return 0.0, 0, 0
    assert N >> 63 == 1
    q = N >> 11
    rest = (N & 0x3FF) | sticky
    q += ((N >> 10) & 1) & ((1 if rest else 0) | (q & 1))
    be = P + e + 1023
    sbit = int(sv != neg) << 63
    bits = (sbit + (((be - 1) << 52) & m64) + q) & m64
    if be > 2046:
        bits = sbit | 0x7FF0000000000000
    sh = min(max(1 - be, 1), 63)
    ms, rem, half = q >> sh, q & ((1 << sh) - 1), 1 << (sh - 1)
    msub = ms + (1 if (rem > half or (rem == half and (ms & 1))) else 0) if (1 - be < 64) else 0
    if be < 1:
        bits = sbit | msub
    return struct.unpack('<d', struct.pack('<Q', bits))[0], q, P


def test_combination_rounds_once_to_nearest_even():
    """Against exact rational rounding (Python's float of a Fraction is correctly
    rounded): random operands, cancellation, exact ties at every shift, every length of
    the high word (both justifications of the 64-bit word, both signs)."""
    import random
    rnd = random.Random(3)
    cases = []
    for _ in range(20000):
        hi, lo = rnd.randint(-2 ** 46, 2 ** 46), rnd.randint(-2 ** 46, 2 ** 46)
        cases.append((hi, lo))
        small = rnd.randint(-2 ** 18, 2 ** 18)
        cases.append((small, -small * 2 ** 28 + rnd.randint(-5, 5)))          # cancellation
        cases.append((rnd.randint(2 ** 40, 2 ** 46), rnd.choice([1, -1]) * 2 ** rnd.randint(0, 40)))  # ties
        cases.append((0, rnd.randint(-2 ** 46, 2 ** 46)))
    for bits in range(1, 47):               # every length of H, with ties and near-ties in L
        for _ in range(40):
            H = rnd.randint(2 ** (bits - 1), 2 ** bits - 1) * rnd.choice([1, -1])
            drop = max(bits + 28 - 53, 0)   # bits of |V| below the rounding point
            L = rnd.randint(0, 2 ** 28 - 1)
            if drop and rnd.random() < 0.5:
                L = (L >> drop << drop) | (1 << (drop - 1)) | rnd.choice([0, 0, 1])
            cases.append((H, L))
            cases.append((H, -L))
    for hi, lo in cases:
        e, neg = rnd.randint(-100, 40), rnd.random() < 0.5
        V = hi * 2 ** 28 + lo
        ref = float(Fraction(V) * Fraction(2) ** e) * (-1 if neg else 1) if V else 0.0
        assert _to_double(hi, lo, e, neg)[0] == ref, (hi, lo, e, neg)


def test_combination_outside_the_normal_range():
    """Beyond the largest double: infinity.  Below the smallest normal: the 53-bit q rounded
    once more to nearest even (the subnormal grid), i.e. Python's correctly rounded float of
    q 2^(P - 52 + e), down to zero."""
    import math
    import random
    rnd = random.Random(8)
    for _ in range(20000):
        hi, lo = rnd.randint(-2 ** 46, 2 ** 46), rnd.randint(-2 ** 46, 2 ** 46)
        if hi == 0 and lo == 0:
            continue
        neg = rnd.random() < 0.5
        _, q, P = _to_double(hi, lo, 0, neg)
        sign = -1.0 if ((hi * 2 ** 28 + lo < 0) != neg) else 1.0
        e_hi = rnd.randint(2047 - 1023 - P, 2047 - 1023 - P + 30)       # be >= 2047
        got = _to_double(hi, lo, e_hi, neg)[0]
        assert math.isinf(got) and math.copysign(1.0, got) == sign
        e_lo = rnd.randint(-1023 - P - 60, -1023 - P)                   # be <= 0
        got = _to_double(hi, lo, e_lo, neg)[0]
        ref = sign * float(Fraction(q) * Fraction(2) ** (P - 52 + e_lo))
        assert got == ref, (hi, lo, e_lo, neg, got, ref)


def _to_double_normal(hi, lo, e, neg):
    """The combination's form for results known to be normal numbers: the same justification
    and rounding as _to_double, and the biased exponent added without the range-end selects."""
    import struct
    m64 = (1 << 64) - 1
    _, q, P = _to_double(hi, lo, 0, False)          # q and P do not depend on e or the sign
    V = hi * 2 ** 28 + lo
    if V == 0:
        return 0.0
    sbit = int((V < 0) != neg) << 63
    bits = (sbit + ((P + e + 1022) << 52) + q) & m64
    return struct.unpack('<d', struct.pack('<Q', bits))[0]


def _combination_input_bounds(K=512):
    """Largest |hi| and |lo| the combination can see in one K chunk: group G sums over k the
    products of digits i + j = G, |t_0| <= 128 and |t_i| <= 64 (i >= 1); hi = v0 2^21 + v1 2^14 +
    v2 2^7 + v3 and lo likewise from v4 .. v7 (an fp32 group sum of G = 6, 7 may round, by less
    than one unit of its last place, which the margin below covers)."""
    tmax = [128] + [64] * 7
    v = [K * sum(tmax[i] * tmax[G - i] for i in range(G + 1) if G - i < 8) for G in range(8)]
    hi = v[0] * 2 ** 21 + v[1] * 2 ** 14 + v[2] * 2 ** 7 + v[3]
    lo = v[4] * 2 ** 21 + v[5] * 2 ** 14 + v[6] * 2 ** 7 + v[7]
    return hi, lo


def test_normal_range_form_gives_the_same_bits():
    """Where the tile's exponent fields keep P + e + 1023 in 1 .. 2046 for every leading-bit
    position P in 0 .. 74, the select-free form returns the general form's bits, a carry of the
    rounding into the exponent included (up to infinity at the top of the range).  The premise
    P <= 74 holds for every value a K = 512 chunk can produce: |V| = |hi 2^28 + lo| stays below
    2^73 by the digit bounds (the conversion's general input range, |H| < 2^47, would not
    ensure it by itself)."""
    import math
    import random
    rnd = random.Random(11)
    hmax, lmax = _combination_input_bounds()
    assert hmax * 2 ** 28 + lmax < 2 ** 73
    for _ in range(20000):
        hi, lo = rnd.randint(-hmax, hmax), rnd.randint(-lmax, lmax)
        if rnd.random() < 0.3:                       # all-ones significands: the rounding carries
            hi, lo = rnd.choice([1, -1]) * (2 ** rnd.randint(1, 44) - 1), 2 ** 28 - 1
        neg = rnd.random() < 0.5
        # the tile condition: e + 1023 >= 1 and e + 1023 + 74 <= 2046
        e = rnd.randint(1 - 1023, 2046 - 1023 - 74)
        a = _to_double(hi, lo, e, neg)[0]
        b = _to_double_normal(hi, lo, e, neg)
        assert (a == b and math.copysign(1.0, a) == math.copysign(1.0, b)) or (math.isnan(a) and math.isnan(b)), \
            (hi, lo, e, neg, a, b)
    # at the ends of the condition the two forms still agree
    for e in (1 - 1023, 2046 - 1023 - 74):
        for hi, lo in ((1, 0), (0, 1), (hmax, lmax), (-hmax, -lmax), (2 ** 44 - 1, 2 ** 28 - 1)):
            assert _to_double(hi, lo, e, False)[0] == _to_double_normal(hi, lo, e, False)
