"""The rounding that ends every exact correlation: an integer T (|T| < 2^112)
becomes the double-float (RN(T), RN(T - RN(T))) 2^-96 with ties to even.
The device's conversion (aqmp_selftest_round, the function the separable
kernels call) is compared bit for bit with that rounding carried out in
Python integers. The cases are random values of every bit length, and
constructed ties at both rounding steps (odd and even 24-bit heads, a
remainder of exactly half a unit, half a unit plus one)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2605_09190_gb300 import aqmp, build_lib
    build_lib.build()
    aqmp.load_library()
    assert torch.cuda.is_available()
    return aqmp


def _rn24(x: int) -> int:
    """x rounded to 24 significant bits, ties to even (x an integer)."""
    if x == 0:
        return 0
    s = -1 if x < 0 else 1
    a = abs(x)
    shift = a.bit_length() - 24
    if shift <= 0:
        return x
    q, r = divmod(a, 1 << shift)
    half = 1 << (shift - 1)
    if r > half or (r == half and q & 1):
        q += 1
    return s * (q << shift)


def _expected(T: int):
    hi = _rn24(T)
    lo = _rn24(T - hi)
    to_f = lambda v: np.float32(np.ldexp(float(v), -96))       # exact: 24 bits, normal range
    return to_f(hi), to_f(lo)


def _cases(rng):
    vals = [0, 1, -1, (1 << 24) - 1, 1 << 24, (1 << 24) + 1, (1 << 25) + 1, (1 << 25) + 3,
            (1 << 111) - 1, -((1 << 111) - 1), 1 << 96, -(1 << 96)]
    for bits in range(1, 112):
        for _ in range(40):
            v = int(rng.integers(0, 1 << 62)) << 50 | int(rng.integers(0, 1 << 50))
            v >>= 112 - bits
            vals.append(v if rng.integers(0, 2) else -v)
    # ties at the first step: a 24-bit head, then exactly half a unit
    for bits in (26, 40, 63, 64, 65, 80, 100, 111):
        shift = bits - 24
        for head in ((1 << 23) + 5, (1 << 23) + 6, (1 << 24) - 1):
            for tail in (1 << (shift - 1), (1 << (shift - 1)) + 1, (1 << (shift - 1)) - 1):
                v = (head << shift) + tail
                vals += [v, -v]
    # ties at the second step: the remainder after the head is itself a
    # 24-bit value followed by exactly half a unit
    for bits in (60, 80, 100, 111):
        shift = bits - 24
        rs = shift - 26                  # the remainder stays below 2^(shift - 2): the head rounds down
        for r_head in ((1 << 23) + 3, (1 << 23) + 4):
            rem = (r_head << rs) + (1 << (rs - 1))
            assert _rn24(rem) - rem in (1 << (rs - 1), -(1 << (rs - 1)))     # a tie
            v = (((1 << 23) + 9) << shift) + rem
            assert _rn24(v) == ((1 << 23) + 9) << shift
            vals += [v, -v]
    return vals


def test_int128_to_double_float_is_correctly_rounded(lib):
    rng = np.random.default_rng(7)
    vals = _cases(rng)
    words = np.zeros((len(vals), 2), np.int64)
    for i, v in enumerate(vals):
        u = v & ((1 << 128) - 1)
        words[i, 0] = np.int64(np.uint64(u & ((1 << 64) - 1)).astype(np.int64))
        words[i, 1] = np.int64(np.uint64(u >> 64).astype(np.int64))
    got = lib.aqmp_selftest_round(torch.from_numpy(words).cuda()).cpu().numpy()
    exp = np.array([_expected(v) for v in vals], np.float32)
    # a zero low word may carry the sign of T (-0.0): the same value; x + 0
    # folds both zeros to +0.0 and leaves every other float as it is
    got = got + np.float32(0.0)
    exp = exp + np.float32(0.0)
    bad = np.nonzero((got.view(np.uint32) != exp.view(np.uint32)).any(axis=1))[0]
    assert bad.size == 0, [(vals[i], got[i], exp[i]) for i in bad[:5]]
