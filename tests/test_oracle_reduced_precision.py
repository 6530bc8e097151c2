"""Pins of the oracle's reduced-precision vector arithmetic against exact
rational arithmetic.

Each step of Alg. 3 that the oracle carries out in binary32 or binary16
(reading R7: FP16 quantities are computed in FP32 and rounded once to FP16;
FP32 ones in FP32; the SpMV accumulates in u_r with one fma per entry) is
recomputed here from its definition with ``fractions.Fraction`` -- every
product and sum exact -- and one correctly rounded conversion where the
definition rounds.  The rounding function below is written from the IEEE 754
definition (round to nearest, ties to even) on exact rationals; it shares
nothing with the oracle's own ``round_to_format``, which works on binary64
values with ``nearbyint``.  Results are compared bit for bit, on random
operands with spread exponents and on crafted ties, so that the plausible
mistakes -- accumulating in FP64 and rounding once, dropping a rounding of
beta or alpha to binary32, rounding y in the wrong precision, a missing
conversion of p_{k-1} to the new u_z -- each fail a test here.

Steps covered: the scaled residual y = round_uz(fl_ur(omega r)) and the Jacobi
z = round_uz(dinv_uz y) (Alg. 3 scaling and preconditioning), the search
direction p = round_uz(fma32(beta32, p, z)), the updates x += alpha p (FP64)
and r = round_ur(fma32(-alpha32, q, r)), the SpMV row sums in FP64, FP32 and
FP16, and the FP64 inner product."""
from fractions import Fraction as F

import numpy as np
import pytest

import oracle


def rne(x: F, p: int, emin: int, emax: int) -> F:
    """Round the exact rational x to the binary format with p significand bits
    (hidden bit included), minimum normal exponent emin and maximum exponent
    emax: round to nearest, ties to the even significand; subnormals keep the
    spacing 2^(emin-p+1); magnitudes that round beyond the largest finite
    value give an infinity (returned as None)."""
    if x == 0:
        return F(0)
    sign = -1 if x < 0 else 1
    a = abs(x)
    e = a.numerator.bit_length() - a.denominator.bit_length()   # 2^e <= a < 2^(e+2)
    while F(2) ** e > a:
        e -= 1
    while F(2) ** (e + 1) <= a:
        e += 1
    e = max(e, emin)
    quantum = F(2) ** (e - p + 1)
    t = a / quantum
    n = t.numerator // t.denominator
    rem = t - n
    if rem > F(1, 2) or (rem == F(1, 2) and n % 2 == 1):
        n += 1
    res = n * quantum
    maxfin = (2 - F(2) ** (1 - p)) * F(2) ** emax
    if res > maxfin:
        return None
    return sign * res


def R64(x):
    return rne(x, 53, -1022, 1023)


def R32(x):
    return rne(x, 24, -126, 127)


def R16(x):
    return rne(x, 11, -14, 15)


RND = {oracle.FP64: R64, oracle.FP32: R32, oracle.FP16: R16}


def fl(v) -> float:
    """A rational that is a binary64 value, as a float (exact)."""
    f = float(v)
    assert F(f) == v
    return f


def same_bits(got, want):
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray([fl(w) for w in want], dtype=np.float64)
    bad = np.nonzero(got.view(np.uint64) != want.view(np.uint64))[0]
    assert bad.size == 0, f"{bad.size} mismatches, first at {bad[0]}: {got[bad[0]]!r} != {want[bad[0]]!r}"


def spread(rng, n, lo=-12, hi=12):
    """Normal values times powers of two in [2^lo, 2^hi]: products and sums of
    these meet every alignment case of the fma."""
    return rng.standard_normal(n) * np.exp2(rng.integers(lo, hi + 1, n).astype(np.float64))


def in_prec(prec, v):
    return oracle.round_to(prec, v)


# --- the rounding function itself, against NumPy's casts --------------------

def test_rne_matches_numpy_casts():
    rng = np.random.default_rng(0)
    v = np.concatenate([spread(rng, 3000, -30, 20), spread(rng, 500, -160, -120)])
    for x in v:
        assert fl(R32(F(x))) == float(np.float32(x))
    for x in spread(rng, 3000, -26, 17):
        h = R16(F(x))
        with np.errstate(over="ignore"):
            want = np.float16(x)
        if np.isinf(want):
            assert h is None
        else:
            assert fl(h) == float(want)


# --- scaling and preconditioning -------------------------------------------

def _diag_matrix(d):
    n = d.size
    return np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32), d


@pytest.mark.parametrize("ur", [oracle.FP64, oracle.FP32])
@pytest.mark.parametrize("uz", [oracle.FP64, oracle.FP32, oracle.FP16])
@pytest.mark.parametrize("omega", [2.0 ** -7, 1.0 / 3.7, 1.0])
def test_scaled_residual_is_one_multiply_in_ur_stored_in_uz(uz, ur, omega):
    rng = np.random.default_rng(11 + 3 * uz + ur)
    n = 2000
    r = in_prec(ur, spread(rng, n, -8, 2))
    rp, ci, d = _diag_matrix(np.ones(n))
    y = oracle.scale_precond(rp, ci, d, oracle.M_NONE, uz, ur, omega, r)
    if ur == oracle.FP64:
        want = [RND[uz](R64(F(omega) * F(ri))) for ri in r]
    else:
        om32 = R32(F(omega))
        want = [RND[uz](R32(om32 * F(ri))) for ri in r]
    same_bits(y, want)


@pytest.mark.parametrize("ur", [oracle.FP64, oracle.FP32])
@pytest.mark.parametrize("uz", [oracle.FP64, oracle.FP32, oracle.FP16])
def test_jacobi_is_one_rounding_of_dinv_times_y(uz, ur):
    rng = np.random.default_rng(40 + 3 * uz + ur)
    n = 1500
    diag = np.exp(rng.uniform(-6, 6, n))
    r = in_prec(ur, spread(rng, n, -6, 2))
    omega = 2.0 ** -3
    rp, ci, d = _diag_matrix(diag)
    z = oracle.scale_precond(rp, ci, d, oracle.M_JACOBI, uz, ur, omega, r)
    want = []
    for ri, ai in zip(r, diag):
        dinv = RND[uz](R64(F(1) / F(ai)))
        y = RND[uz](R64(F(omega) * F(ri)) if ur == oracle.FP64 else R32(R32(F(omega)) * F(ri)))
        want.append(R64(dinv * y) if uz == oracle.FP64 else RND[uz](R32(dinv * y)))
    same_bits(z, want)


# --- search direction ---------------------------------------------------------

def _direction_ref(uz, beta, z, pprev):
    out = []
    for zi, pi in zip(z, pprev):
        pold = RND[uz](F(pi))
        if uz == oracle.FP64:
            out.append(R64(F(beta) * pold + F(zi)))
        else:
            out.append(RND[uz](R32(R32(F(beta)) * pold + F(zi))))
    return out


@pytest.mark.parametrize("uz", [oracle.FP64, oracle.FP32, oracle.FP16])
@pytest.mark.parametrize("pprec", [oracle.FP64, oracle.FP32, oracle.FP16])
def test_direction_random(uz, pprec):
    rng = np.random.default_rng(70 + 3 * uz + pprec)
    n = 3000
    z = in_prec(uz, spread(rng, n, -10, 4))
    pprev = in_prec(pprec, spread(rng, n, -10, 4))
    beta = float(rng.uniform(0.05, 1.7))
    same_bits(oracle.direction(uz, False, beta, z, pprev), _direction_ref(uz, beta, z, pprev))


def test_direction_crafted_ties():
    # fp16: 1 + beta*2^-10 with beta = 0.5 is the binary16 midpoint 1 + 2^-11
    # (ties to even: 1); beta = 1 + 2^-19 with p = 2^-11 makes the exact value
    # 1 + 2^-11 + 2^-30, which binary32 rounds to the midpoint (then 1), while
    # a single rounding to binary16 would give 1 + 2^-10
    z = np.array([1.0, 1.0, 1.0, -1.0, 3.0])
    p = np.array([2.0 ** -10, 2.0 ** -11, 2.0 ** -11, -(2.0 ** -11), 2.0 ** -9])
    for beta in (0.5, 1.0 + 2.0 ** -19, 1.0 + 2.0 ** -40):
        got = oracle.direction(oracle.FP16, False, beta, z, p)
        same_bits(got, _direction_ref(oracle.FP16, beta, z, p))
    got = oracle.direction(oracle.FP16, False, 1.0 + 2.0 ** -19, z[1:2], p[1:2])
    assert got[0] == 1.0
    # beta not representable in binary32: the binary32 rounding of beta matters
    beta = 1.0 + 2.0 ** -30
    zz = np.array([0.0])
    pp = np.array([1.0])
    assert oracle.direction(oracle.FP32, False, beta, zz, pp)[0] == 1.0


def test_direction_first_iteration_copies_z():
    z = np.array([0.5, -2.0, 3.25])
    assert np.array_equal(oracle.direction(oracle.FP16, True, 7.0, z, np.full(3, 9.0)), z)


# --- x and r updates ------------------------------------------------------------

@pytest.mark.parametrize("ur", [oracle.FP64, oracle.FP32])
@pytest.mark.parametrize("pprec", [oracle.FP64, oracle.FP32, oracle.FP16])
def test_updates(ur, pprec):
    rng = np.random.default_rng(90 + 3 * ur + pprec)
    n = 3000
    p = in_prec(pprec, spread(rng, n, -8, 3))
    q = in_prec(ur, spread(rng, n, -8, 3))
    x = spread(rng, n, -4, 4)
    r = in_prec(ur, spread(rng, n, -10, 0))
    alpha = float(rng.uniform(0.1, 3.0))
    x1, r1 = oracle.update_xr(ur, alpha, p, q, x, r)
    same_bits(x1, [R64(F(alpha) * F(pi) + F(xi)) for pi, xi in zip(p, x)])
    if ur == oracle.FP64:
        want = [R64(-F(alpha) * F(qi) + F(ri)) for qi, ri in zip(q, r)]
    else:
        a32 = R32(F(alpha))
        want = [R32(-a32 * F(qi) + F(ri)) for qi, ri in zip(q, r)]
    same_bits(r1, want)


def test_update_r32_alpha_rounded_to_binary32():
    # alpha = 1 + 2^-30 is 1 in binary32: r - alpha q must be exactly r - q
    q = np.array([1.0, 2.0 ** -3])
    r = np.array([1.0, 1.0])
    _, r1 = oracle.update_xr(oracle.FP32, 1.0 + 2.0 ** -30, np.zeros(2), q, np.zeros(2), r)
    assert r1[0] == 0.0 and r1[1] == 1.0 - 2.0 ** -3


# --- SpMV row sums ----------------------------------------------------------------

def _random_csr(rng, n, maxw):
    lens = rng.integers(1, maxw + 1, n)
    rowptr = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
    col = np.concatenate([np.sort(rng.choice(n, size=k, replace=False)) for k in lens]).astype(np.int32)
    return rowptr, col


def _tie_rows():
    # rows whose partial sums sit exactly on binary32 / binary16 midpoints:
    # per-entry rounding (ties to even) keeps 1 where one final rounding of
    # the FP64 sum would not
    vals = [[1.0, 2.0 ** -12, 2.0 ** -12], [1.0, 2.0 ** -24, 2.0 ** -24, 2.0 ** -24],
            [-1.0, -(2.0 ** -25), 2.0 ** -50], [1.0, 2.0 ** -6, 2.0 ** -6]]
    return vals


def _rowsum_ref(prec, rowptr, col, aval, p):
    out = []
    for i in range(rowptr.size - 1):
        acc = F(0)
        for k in range(rowptr[i], rowptr[i + 1]):
            if prec == oracle.FP64:
                acc = R64(F(aval[k]) * F(p[col[k]]) + acc)
            else:
                acc = R32(F(aval[k]) * RND[prec](F(p[col[k]])) + acc)
        out.append(RND[prec](acc))
    return out


@pytest.mark.parametrize("prec", [oracle.FP64, oracle.FP32, oracle.FP16])
@pytest.mark.parametrize("pprec", [oracle.FP64, oracle.FP16])
def test_spmv_row_sum_is_an_fma_chain_in_u(prec, pprec):
    rng = np.random.default_rng(120 + 3 * prec + pprec)
    n = 500
    rowptr, col = _random_csr(rng, n, 12)
    lo = -6 if prec == oracle.FP16 else -14
    aval = in_prec(prec, spread(rng, col.size, lo, 4))
    p = in_prec(pprec, spread(rng, n, lo, 4))
    q = oracle.spmv(rowptr, col, aval, prec, p)
    same_bits(q, _rowsum_ref(prec, rowptr, col, aval, p))


@pytest.mark.parametrize("prec", [oracle.FP32, oracle.FP16])
def test_spmv_crafted_ties(prec):
    rows = _tie_rows()
    n = max(len(r) for r in rows)
    rowptr = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int32)
    col = np.concatenate([np.arange(len(r)) for r in rows]).astype(np.int32)
    aval = in_prec(prec, np.concatenate(rows))
    p = np.ones(n)
    q = oracle.spmv(rowptr, col, aval, prec, p)
    same_bits(q, _rowsum_ref(prec, rowptr, col, aval, p))
    if prec == oracle.FP32:
        assert q[0] == 1.0 + 2.0 ** -11 and q[1] == 1.0


@pytest.mark.parametrize("lo,hi", [(-20, 20), (0, 0)])
def test_dot_is_a_recursive_binary64_sum(lo, hi):
    # (0, 0): terms of one magnitude, where rounding each product before the
    # add (no fma contraction) changes the sum's rounding every ~100 terms
    rng = np.random.default_rng(7 + abs(lo))
    a, b = spread(rng, 4000, lo, hi), spread(rng, 4000, lo, hi)
    s = F(0)
    for ai, bi in zip(a, b):
        s = R64(s + R64(F(ai) * F(bi)))
    assert oracle.dot(a, b) == fl(s)
