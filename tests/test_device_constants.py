"""Constants typed into the CUDA sources agree with their definitions.

theta_m are Higham (2005), Table 2.3 (the oracle types the same published
values independently); the Pade numerator coefficients and the leading
backward-error coefficient |c_27| of the [13/13] approximant follow from
their closed forms."""
import math
import os
import re
from fractions import Fraction

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "paper_2603_15964_gb300", "csrc", "lmep_device.cuh")


def source():
    with open(SRC) as f:
        return f.read()


def test_log2_c27():
    v = float(re.search(r"LOG2_C27\s*=\s*(-?[0-9.]+)f", source()).group(1))
    c27 = Fraction(math.factorial(13) ** 2, math.factorial(26) * math.factorial(27))
    assert abs(v - math.log2(c27)) < 1e-3


def test_log2_theta13_is_rounded_down():
    v = float(re.search(r"const float lt = ([0-9.]+)f", source()).group(1))
    th = float(re.search(r"THETA13 = ([0-9.e+-]+);", source()).group(1))
    assert v <= math.log2(th) and math.log2(th) - v < 1e-5


def test_thetas_match_higham_table():
    text = source()
    want = {3: 1.495585217958292e-2, 5: 2.539398330063230e-1, 7: 9.504178996162932e-1,
            9: 2.097847961257068e0, 13: 5.371920351148152e0}
    for m, v in want.items():
        got = float(re.search(rf"THETA{m} = ([0-9.e+-]+);", text).group(1))
        assert got == v


def test_pade_recurrence_matches_closed_form():
    """b_{j+1} = b_j (m - j) / ((2m - j)(j + 1)) is the ratio of (2m-j)! m! / ((2m)! j! (m-j)!)."""
    for m in (3, 5, 7, 9, 13):
        b = Fraction(1)
        for j in range(m):
            b = b * (m - j) / ((2 * m - j) * (j + 1))
            closed = Fraction(math.factorial(2 * m - j - 1) * math.factorial(m),
                              math.factorial(2 * m) * math.factorial(j + 1) * math.factorial(m - j - 1))
            assert b == closed


def test_no_ell_correction_below_theta13():
    """The kernel skips the 2009 ell estimate when ||X||_1 <= theta_13.  That is
    exact because ||(|X|)^27||_1 / ||X||_1 <= ||X||_1^26, so the ell argument
    |c27| ||X||_1^26 stays below u = 2^-53 up to ||X||_1 = 5.43 > theta_13."""
    th = float(re.search(r"THETA13 = ([0-9.e+-]+);", source()).group(1))
    c27 = Fraction(math.factorial(13) ** 2, math.factorial(26) * math.factorial(27))
    bound = math.log2(c27) + 26 * math.log2(th)
    assert bound < -53
    limit = 2 ** ((-53 - math.log2(c27)) / 26)
    assert 5.42 < limit < 5.44 and th < limit
