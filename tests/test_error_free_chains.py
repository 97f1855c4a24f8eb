"""The short error-free chains of the FP64-class residual kernels, modelled in
exact rational arithmetic.

The residual kernels sum each short run of products a_k b_k (complex64 data)
with a biased accumulator: sigma is the least power of two >= 2 (1 + 2^-17)
(sum |a|_1) (max |b|_inf), tau starts at sigma, and every step is

    tau' = fma(a, b, tau);  q = tau' - tau;  r += fma(a, b, -q)

so that the run's sum is (tau - sigma) + r.  This is the ExtractScalar step of
Rump, Ogita & Oishi ("Accurate floating-point summation part I: faithful
rounding", SIAM J. Sci. Comput. 31(1), 2008) applied through the FMA.  The
model below rounds every FP32 operation exactly (round to nearest, ties to
even, with subnormals) and checks what the kernels rely on:
  * q = tau' - tau is exact at every step, and tau stays within [1/2, 3/2] sigma;
  * tau - sigma is exact;
  * the sum's error stays within 2^-39 of sum |a_k b_k| (typically 1.5-6 units
    of 2^-48: each remainder is rounded once on a grid of about 2^-23 sigma,
    and sigma is 5-15 times the terms' size), 10^4 times and more below plain
    FP32 summation.  Dot2 (Ogita, Rump & Oishi 2005), modelled alongside, stays
    within a few units of 2^-48: the chains trade about 5 bits of the block
    sums for 2.5 times fewer operations.
"""
from fractions import Fraction as F

import numpy as np
import pytest

EMIN = -126      # smallest normal exponent of binary32


def f32(x):
    """x (a Fraction) rounded to the nearest binary32 value, ties to even."""
    if x == 0:
        return F(0)
    s = -1 if x < 0 else 1
    x = abs(x)
    e = x.numerator.bit_length() - x.denominator.bit_length()
    if F(2) ** e > x:
        e -= 1
    e = max(e, EMIN)                       # subnormals share the grid of 2^-126
    ulp = F(2) ** (e - 23)
    m = x / ulp
    lo = m.numerator // m.denominator
    rem = m - lo
    if rem > F(1, 2) or (rem == F(1, 2) and lo % 2 == 1):
        lo += 1
    assert lo <= 2 ** 24
    return s * lo * ulp


def fma(a, b, c):
    return f32(a * b + c)


def add(a, b):
    return f32(a + b)


def sub(a, b):
    return f32(a - b)


def pow2_ceil(v):
    """The least power of two >= v for v > 0 (2^-126 for subnormals), 0 for 0."""
    if v == 0:
        return F(0)
    e = EMIN
    while F(2) ** e < v:
        e += 1
    return F(2) ** e


MARGIN = F(2) + F(2) ** -16     # 2 (1 + 2^-17), exact in binary32


def chain_sigma(sa, mb):
    return pow2_ceil(f32(f32(MARGIN * sa) * mb))


def real_chain(terms, sigma, check=True):
    """(tau - sigma, r) of a biased chain over real terms (a, b)."""
    tau, r = sigma, F(0)
    for a, b in terms:
        t2 = fma(a, b, tau)
        q = sub(t2, tau)
        if check:
            assert q == t2 - tau                                   # Sterbenz: exact
            assert sigma / 2 <= t2 <= F(3, 2) * sigma or sigma == 0
        r = add(r, fma(a, b, -q))
        tau = t2
    S = sub(tau, sigma)
    if check:
        assert S == tau - sigma
    return S, r


def complex_chain(a, b):
    """sum_k a_k b_k for complex64 a, b (lists of (re, im) Fractions), as the
    kernels run it: one sigma for the real and the imaginary chain."""
    sa = F(0)
    for ar, ai in a:
        sa = add(sa, add(abs(ar), abs(ai)))
    mb = max(max(abs(br), abs(bi)) for br, bi in b)
    sigma = chain_sigma(sa, mb)
    re_terms, im_terms = [], []
    for (ar, ai), (br, bi) in zip(a, b):
        re_terms += [(ar, br), (-ai, bi)]
        im_terms += [(ar, bi), (ai, br)]
    Sr, rr = real_chain(re_terms, sigma)
    Si, ri = real_chain(im_terms, sigma)
    return (Sr + rr, Si + ri)


def two_sum(a, b):
    s = add(a, b)
    bb = sub(s, a)
    return s, add(sub(a, sub(s, bb)), sub(b, bb))


def dot2_real(terms):
    """Dot2: every product split exactly (p + ep), every sum compensated."""
    hi, lo = F(0), F(0)
    for a, b in terms:
        p = f32(a * b)
        ep = fma(a, b, -p)
        hi, q = two_sum(hi, p)
        lo = add(lo, add(q, ep))
    return hi + lo


def dot2_complex(a, b):
    re_terms, im_terms = [], []
    for (ar, ai), (br, bi) in zip(a, b):
        re_terms += [(ar, br), (-ai, bi)]
        im_terms += [(ar, bi), (ai, br)]
    return dot2_real(re_terms), dot2_real(im_terms)


def _c64(rng, n, spread):
    x = (rng.normal(size=n) + 1j * rng.normal(size=n)) * np.exp(spread * rng.normal(size=n))
    return [(F(float(np.float32(v.real))), F(float(np.float32(v.imag)))) for v in x]


def _exact(a, b):
    re = sum(ar * br - ai * bi for (ar, ai), (br, bi) in zip(a, b))
    im = sum(ar * bi + ai * br for (ar, ai), (br, bi) in zip(a, b))
    mag = sum((abs(ar) + abs(ai)) * (abs(br) + abs(bi)) for (ar, ai), (br, bi) in zip(a, b))
    return re, im, mag


@pytest.mark.parametrize("L", [2, 4])
@pytest.mark.parametrize("spread", [0.0, 1.5])
def test_chain_is_exact_where_claimed_and_accurate(L, spread):
    # runs of L complex products (2L real terms per part), as in the kernels:
    # L = 2 for a lane's two columns of a row, 4 for four rows / K indices / rank rows
    rng = np.random.default_rng(10 * L + int(spread))
    units = 2.0 ** -48
    chain, dot2 = [], []
    for _ in range(150):
        a, b = _c64(rng, L, spread), _c64(rng, L, spread)
        re, im, mag = _exact(a, b)
        got_re, got_im = complex_chain(a, b)
        chain.append(float(max(abs(got_re - re), abs(got_im - im)) / mag) / units)
        d_re, d_im = dot2_complex(a, b)
        dot2.append(float(max(abs(d_re - re), abs(d_im - im)) / mag) / units)
    assert max(chain) < 512 and np.median(chain) < 16
    assert max(dot2) < 8


def test_chain_beats_fp32_summation_on_cancelling_sums():
    # sums that cancel to 1e-6 of their terms: FP32 loses about every digit,
    # the chain keeps the result within 2^-39 of sum |a b|
    rng = np.random.default_rng(3)
    worst_chain = worst_fp32 = 0.0
    for _ in range(100):
        a, b = _c64(rng, 4, 0.0), _c64(rng, 4, 0.0)
        re, im, mag = _exact(a, b)
        # shift the last term so that the real part nearly cancels
        ar, ai = a[-1]
        br, bi = b[-1]
        target = -(re - (ar * br - ai * bi)) + F(float(np.float32(1e-6))) * mag
        a[-1] = (f32(target / br + ai * bi / br) if br != 0 else ar, ai)
        re, im, mag = _exact(a, b)
        got_re, _ = complex_chain(a, b)
        plain = F(0)
        for (xr, xi), (yr, yi) in zip(a, b):
            plain = f32(plain + f32(f32(xr * yr) - f32(xi * yi)))
        worst_chain = max(worst_chain, float(abs(got_re - re) / mag))
        worst_fp32 = max(worst_fp32, float(abs(plain - re) / mag))
    assert worst_chain < 512 * 2.0 ** -48
    assert worst_fp32 > 1e4 * worst_chain


def test_chain_edge_cases():
    z = [(F(0), F(0))] * 4
    one = [(F(1), F(0))] * 4
    assert complex_chain(z, one) == (0, 0)                 # sigma = 0: every product is zero
    assert complex_chain(one, z) == (0, 0)
    # exact cancellation to zero
    a = [(F(3), F(0)), (F(-3), F(0))]
    b = [(F(5, 4), F(0)), (F(5, 4), F(0))]
    assert complex_chain(a, b) == (0, 0)
    # a subnormal bound: sigma is the smallest normal power of two, the sum still right
    tiny = F(2) ** -140
    got = complex_chain([(tiny, F(0))], [(F(1, 2), F(0))])
    assert got == (tiny / 2, 0)
    # the bound is met with equality at a power of two: tau still within [1/2, 3/2] sigma
    a = [(F(1), F(0))] * 4
    b = [(F(1), F(0))] * 4
    assert complex_chain(a, b) == (4, 0)


@pytest.mark.parametrize("seed", range(6))
def test_chain_at_the_edge_of_its_bound(seed):
    # every term of one sign and sum |a b| as large as sigma allows (the bound's
    # sigma lands exactly on a power of two), each term with low bits below
    # tau's grid, so that every step rounds: tau must stay >= sigma / 2 and q,
    # tau - sigma exact (real_chain asserts both)
    rng = np.random.default_rng(seed)
    n = 4
    b = [(F(1), F(0))] * n
    v = [f32(F(float(x))) for x in rng.uniform(0.05, 0.11, size=n - 1)]
    sa_rest = F(0)
    for x in v:
        sa_rest = add(sa_rest, x)
    last = f32(1 / MARGIN - sa_rest)

    def ulp(x):
        e = x.numerator.bit_length() - x.denominator.bit_length()
        if F(2) ** e > x:
            e -= 1
        return F(2) ** (e - 23)

    # the largest last term whose chain still gets sigma = 1 (a few float steps at most)
    for _ in range(64):
        if chain_sigma(add(sa_rest, last), F(1)) <= 1:
            break
        last = f32(last - ulp(last))
    for _ in range(64):
        up = f32(last + ulp(last))
        if chain_sigma(add(sa_rest, up), F(1)) > 1:
            break
        last = up
    a = [(-x, F(0)) for x in v + [last]]
    sa = F(0)
    for ar, ai in a:
        sa = add(sa, add(abs(ar), abs(ai)))
    assert chain_sigma(sa, F(1)) == 1
    got_re, got_im = complex_chain(a, b)
    exact = sum(ar for ar, _ in a)
    assert got_im == 0
    assert abs(got_re - exact) <= 2.0 ** -46 * abs(exact)


def test_pow2_ceil_matches_the_bit_trick():
    # the kernels take (bits(v) + 0x7FFFFF) & 0xFF800000; the model's definition agrees
    rng = np.random.default_rng(5)
    vals = np.concatenate([np.float32(2.0) ** np.arange(-149, 127, 7, dtype=np.float32),
                           rng.random(200).astype(np.float32) * np.float32(1e3),
                           np.array([0.0, 1.0, 1.5, 3.0, 1e-40, 1e-45], dtype=np.float32)]).astype(np.float32)
    bits = vals.view(np.uint32)
    trick = ((bits.astype(np.uint64) + 0x007FFFFF) & 0xFF800000).astype(np.uint32).view(np.float32)
    for v, t in zip(vals, trick):
        assert F(float(t)) == pow2_ceil(F(float(v))), v


# ---------------------------------------------------------------------------
# Chains on a common grid (the residual kernels' blocks of up to 64 x 64): every
# chain feeding one output sum takes sigma = pow2_ceil((2 + 2^-10) * bound * mb),
# bound the block's largest row 1-norm (rounded up), mb the largest input
# component; the lanes' grid parts tau - sigma are added in plain FP32 (the kernel
# asserts nothing: the model checks every such addition is exact) and so are the
# remainders.

GRID_MARGIN = F(2) + F(2) ** -10


def grid_sigma(bound, mb):
    return pow2_ceil(f32(f32(GRID_MARGIN * bound) * mb))


def grid_row(a, x, bound, lanes):
    """sum_j a_j x_j for one row (complex64 a, x) split over `lanes` chains (lane l
    takes the terms j with j % lanes == l), as the kernels run it; returns the sum
    and checks the exactness claims."""
    mb = max(max(abs(xr), abs(xi)) for xr, xi in x)
    sigma = grid_sigma(bound, mb)
    parts = []
    for l in range(lanes):
        re_t, im_t = [], []
        for (ar, ai), (xr, xi) in list(zip(a, x))[l::lanes]:
            re_t += [(ar, xr), (-ai, xi)]
            im_t += [(ar, xi), (ai, xr)]
        parts.append((real_chain(re_t, sigma), real_chain(im_t, sigma)))
    out = []
    for c in range(2):
        g, r = F(0), F(0)
        for p in parts:                       # lane order of the warp reduction
            g2 = add(g, p[c][0])
            assert g2 == g + p[c][0]              # grid parts add exactly
            g = g2
            r = add(r, p[c][1])
        out.append(g + r)
    return out


def _bound_ru(rows):
    """largest row 1-norm, rounded up to binary32 (the kernels' FP64 sum, rounded up)"""
    v = max(sum(abs(ar) + abs(ai) for ar, ai in row) for row in rows)
    w = f32(v)
    while w < v:
        w = f32(w + w * F(2) ** -24)
    return w


@pytest.mark.parametrize("spread", [0.0, 1.5])
def test_common_grid_rows_exact_where_claimed_and_accurate(spread):
    # a 16 x 64 block (one row group's share of a 64 x 64 block): each row over 8
    # lanes of 8 columns, sigma from the whole block's bound
    rng = np.random.default_rng(20 + int(spread))
    rows = [_c64(rng, 64, spread) for _ in range(16)]
    x = _c64(rng, 64, spread)
    bound = _bound_ru(rows)
    mb = max(max(abs(xr), abs(xi)) for xr, xi in x)
    sigma = grid_sigma(bound, mb)
    worst = 0.0
    for a in rows:
        re, im, mag = _exact(a, x)
        got = grid_row(a, x, bound, 8)
        worst = max(worst, float(max(abs(got[0] - re), abs(got[1] - im)) / sigma))
    # a few units of 2^-48 sigma per chain step (16 real steps per lane chain)
    assert worst < 64 * 2.0 ** -48


def test_common_grid_keeps_fp64_class_accuracy_on_cancelling_rows():
    # a row whose sum cancels to 1e-7 of its terms: FP32 summation keeps no digit,
    # the common grid keeps the sum within 2^-40 of sigma (sigma ~ 2-4 x the bound)
    rng = np.random.default_rng(7)
    a = _c64(rng, 64, 0.0)
    x = _c64(rng, 64, 0.0)
    re, im, mag = _exact(a, x)
    ar, ai = a[-1]
    xr, xi = x[-1]
    target = -(re - (ar * xr - ai * xi)) + F(float(np.float32(1e-7))) * mag
    a[-1] = (f32((target + ai * xi) / xr), ai)
    re, im, mag = _exact(a, x)
    bound = _bound_ru([a])
    mb = max(max(abs(v), abs(w)) for v, w in x)
    got = grid_row(a, x, bound, 8)
    assert abs(got[0] - re) <= grid_sigma(bound, mb) * F(2) ** -40
    plain = F(0)
    for (p, q), (s, t) in zip(a, x):
        plain = f32(plain + f32(f32(p * s) - f32(q * t)))
    assert abs(plain - re) > 1e3 * abs(got[0] - re)


def test_common_grid_at_the_edge_of_its_bound():
    # every term of one sign, the row's 1-norm equal to the block bound, and 64
    # terms per output: the partial sums reach bound * mb < sigma / 2 and the
    # lane sums must still be exact (grid_row asserts it)
    rng = np.random.default_rng(11)
    vals = [f32(F(float(v))) for v in rng.uniform(0.5, 1.0, size=64)]
    a = [(v, F(0)) for v in vals]
    x = [(F(1), F(0))] * 64
    bound = _bound_ru([a])
    got = grid_row(a, x, bound, 8)
    assert abs(got[0] - sum(vals)) <= grid_sigma(bound, F(1)) * F(2) ** -44
    assert got[1] == 0
    # a bound of zero (a zero block): every sum is zero
    z = [(F(0), F(0))] * 8
    assert grid_row(z, x[:8], F(0), 8) == [0, 0]


def test_common_grid_two_stage_low_rank():
    # a low-rank block's second stage: o_i = sum_l Y_il t_l with t_l = G_l + R_l the
    # first stage's grid sum and remainder; sigma_2 from the bound |G_l| <= sigma_1 / 2
    # (the leading parts through the chain, the trailing parts into r).  The chain's
    # claims hold (real_chain asserts them) and the output is within 2^-38 of sigma_2.
    rng = np.random.default_rng(13)
    k, n = 8, 64
    V = [_c64(rng, n, 0.5) for _ in range(k)]
    x = _c64(rng, n, 0.0)
    bV = _bound_ru(V)
    mb = max(max(abs(p), abs(q)) for p, q in x)
    s1 = grid_sigma(bV, mb)
    t = []
    for row in V:
        g = grid_row(row, x, bV, 32)                  # the kernels' 32-lane stage 1
        re, im, _ = _exact(row, x)
        # 32 lanes' remainders, each up to 2^-22 sigma_1, summed in FP32: a few units of 2^-41
        assert abs(g[0] - re) <= s1 * F(2) ** -38 and abs(g[1] - im) <= s1 * F(2) ** -38
        t.append(g)
    Y = _c64(rng, k, 0.5)                             # one output row of U (rank entries)
    bY = _bound_ru([Y])
    s2 = grid_sigma(bY, s1 / 2)
    # split each t_l into the FP32 leading part the chain takes and the trailing rest
    hi = [(f32(a), f32(b)) for a, b in t]
    lo = [(a - h[0], b - h[1]) for (a, b), h in zip(t, hi)]
    assert max(max(abs(a), abs(b)) for a, b in hi) <= s1 / 2
    re_t, im_t = [], []
    for (yr, yi), (hr, hh) in zip(Y, hi):
        re_t += [(yr, hr), (-yi, hh)]
        im_t += [(yr, hh), (yi, hr)]
    Sr, rr = real_chain(re_t, s2)
    Si, ri = real_chain(im_t, s2)
    got_re = Sr + rr + sum(yr * lr - yi * li for (yr, yi), (lr, li) in zip(Y, lo))
    got_im = Si + ri + sum(yr * li + yi * lr for (yr, yi), (lr, li) in zip(Y, lo))
    ex_re = sum(yr * a - yi * b for (yr, yi), (a, b) in zip(Y, t))
    ex_im = sum(yr * b + yi * a for (yr, yi), (a, b) in zip(Y, t))
    assert abs(got_re - ex_re) <= s2 * F(2) ** -38 and abs(got_im - ex_im) <= s2 * F(2) ** -38
