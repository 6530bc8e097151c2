"""Pins for the precision selector, Eq. (precision_selector), and the two
attainable-accuracy indicators, Eq. (eta_k) and Eq. (linear criterion).

For a geometric residual sequence delta_t = delta_0 rho^t the indicators have
closed forms (finite geometric sums), so the iteration at which u_r switches
to FP32 and the iterations at which u_z steps down follow from logarithms,
independently of the oracle's loops.  A wrong constant (3+C, 2+C, 5+2C), a
wrong eps32, a dropped window term or an off-by-one in the window would move
the predicted switch iteration."""
import math

import numpy as np
import pytest

import oracle

EPS32 = 2.0 ** -24


def _geometric(rho, m, d0=1.0):
    return d0 * rho ** np.arange(m + 1, dtype=np.float64)


def _first(trace, pred):
    idx = [k for k, v in enumerate(trace) if pred(v)]
    return idx[0] if idx else None


def _ceil_away_from_ties(x):
    frac = x - math.floor(x)
    assert 1e-6 < frac < 1 - 1e-6, "parameters too close to a tie"
    return math.ceil(x)


@pytest.mark.parametrize("rho,d,C,tol,nb", [(0.8, 10, 1.0, 1e-10, 1.0), (0.93, 10, 1.0, 1e-10, 37.0),
                                            (0.5, 4, 2.0, 1e-8, 3.0), (0.97, 20, 0.5, 1e-12, 1.0)])
def test_window_switch_iteration_closed_form(rho, d, C, tol, nb):
    m = 3000
    delta = _geometric(rho, m)
    T = tol * nb
    # eta_k for k >= d+1: eps32 (( (3+C)/rho + (2+C) ) delta_0 rho^(k-d) (1-rho^(d+1))/(1-rho)
    amp = EPS32 * ((3 + C) / rho + (2 + C)) * (1 - rho ** (d + 1)) / (1 - rho)
    k_star = d + _ceil_away_from_ties(math.log(T / amp) / math.log(rho))
    assert k_star > d + 1
    pol = oracle.Policy(u0=oracle.FP64, criterion=oracle.WINDOW, d=d, C=C, tau_zs=0.0, tau_zh=0.0)
    tr = oracle.selector_trace(delta, nb, tol, pol)
    got = _first(tr, lambda v: (v & 0xF) == oracle.FP32)
    assert got == k_star
    # the indicator itself against the closed-form sum at a few k
    for k in (d + 1, d + 7, k_star):
        closed = amp * rho ** (k - d)
        assert oracle.eta_window(delta, k, d, C) == pytest.approx(closed, rel=1e-12)


@pytest.mark.parametrize("rho,ell,C,tol,nb", [(0.8, 5, 1.0, 1e-10, 1.0), (0.95, 5, 1.0, 1e-10, 12.0),
                                              (0.6, 3, 2.0, 1e-9, 1.0)])
def test_linear_switch_iteration_closed_form(rho, ell, C, tol, nb):
    m = 3000
    delta = _geometric(rho, m)
    T = tol * nb
    # eta_k = eps32 (5+2C) delta_0 rho^(k-1) / (1 - rho)
    k_star = 1 + _ceil_away_from_ties(math.log(T * (1 - rho) / (EPS32 * (5 + 2 * C))) / math.log(rho))
    k_star = max(k_star, ell)
    pol = oracle.Policy(u0=oracle.FP64, criterion=oracle.LINEAR, ell=ell, C=C, tau_zs=0.0, tau_zh=0.0)
    tr = oracle.selector_trace(delta, nb, tol, pol)
    assert _first(tr, lambda v: (v & 0xF) == oracle.FP32) == k_star
    k = k_star
    assert oracle.eta_linear(delta, k, ell, C) == pytest.approx(
        EPS32 * (5 + 2 * C) * rho ** (k - 1) / (1 - rho), rel=1e-12)


def test_indicators_undefined_before_window():
    delta = _geometric(0.1, 30)
    for k in range(10):
        assert math.isinf(oracle.eta_window(delta, k, 10, 1.0))
    assert math.isfinite(oracle.eta_window(delta, 10, 10, 1.0))
    for k in range(5):
        assert math.isinf(oracle.eta_linear(delta, k, 5, 1.0))
    # a residual that does not decrease gives no estimate
    flat = np.ones(20)
    assert math.isinf(oracle.eta_linear(flat, 10, 5, 1.0))


@pytest.mark.parametrize("rho", [0.9, 0.77])
def test_uz_thresholds_closed_form(rho):
    m = 400
    delta = _geometric(rho, m)
    pol = oracle.Policy(u0=oracle.FP64, criterion=oracle.WINDOW, tau_zs=1e-4, tau_zh=1e-6)
    tr = oracle.selector_trace(delta, 1.0, 1e-300, pol)   # u_r never switches
    k32 = math.floor(math.log(1e-4) / math.log(rho)) + 1   # first k with rho^k < 1e-4
    k16 = math.floor(math.log(1e-6) / math.log(rho)) + 1
    assert _first(tr, lambda v: (v >> 4) == oracle.FP32) == k32
    assert _first(tr, lambda v: (v >> 4) == oracle.FP16) == k16
    assert all((v & 0xF) == oracle.FP64 for v in tr)
    # u0 caps the precision from above: AMP-PCG(FP16) is FP16 from the start
    pol16 = oracle.Policy(u0=oracle.FP16, criterion=oracle.WINDOW)
    assert all((v >> 4) == oracle.FP16 for v in oracle.selector_trace(delta, 1.0, 1e-300, pol16))
    pol32 = oracle.Policy(u0=oracle.FP32, criterion=oracle.WINDOW)
    tr32 = oracle.selector_trace(delta, 1.0, 1e-300, pol32)
    assert _first(tr32, lambda v: (v >> 4) == oracle.FP16) == k16
    assert (tr32[0] >> 4) == oracle.FP32


def test_selector_latch_and_fixed():
    nu = np.array([1.0, 1e-5, 1e-3, 1e-7, 1e-5])
    free = oracle.Policy(u0=oracle.FP64, criterion=oracle.WINDOW, latch=0)
    tr = oracle.selector_trace(nu, 1.0, 1e-300, free)
    assert [v >> 4 for v in tr] == [0, 1, 0, 2, 1]
    latched = oracle.Policy(u0=oracle.FP64, criterion=oracle.WINDOW, latch=1)
    tr = oracle.selector_trace(nu, 1.0, 1e-300, latched)
    assert [v >> 4 for v in tr] == [0, 1, 1, 2, 2]
    fixed = oracle.Policy(criterion=oracle.FIXED, fixed_uz=oracle.FP16, fixed_ur=oracle.FP32)
    assert all(v == (2 << 4 | 1) for v in oracle.selector_trace(nu, 1.0, 1e-10, fixed))


def test_select_pure_function():
    # Eq. (precision_selector) case by case
    assert oracle.select(1e-3, oracle.FP64, 1e-4, 1e-6, 1.0, 0.5) == (oracle.FP64, oracle.FP64)
    assert oracle.select(1e-5, oracle.FP64, 1e-4, 1e-6, 1.0, 0.5) == (oracle.FP32, oracle.FP64)
    assert oracle.select(1e-7, oracle.FP64, 1e-4, 1e-6, 0.5, 0.5) == (oracle.FP16, oracle.FP32)
    assert oracle.select(1e-4, oracle.FP64, 1e-4, 1e-6, 0.6, 0.5) == (oracle.FP64, oracle.FP64)
    assert oracle.select(1e-6, oracle.FP16, 1e-4, 1e-6, 0.4, 0.5) == (oracle.FP16, oracle.FP32)


def test_scale_linf_pow2():
    for m in [1.0, 0.75, 0.5, 3.0, 2.0 ** -30, 1e-10, 7e5, 2.0 ** 20]:
        w = oracle.scale(oracle.SCALE_LINF_POW2, 1.0, m)
        assert math.frexp(w)[0] == 0.5                      # a power of two
        assert 0.5 < w * m <= 1.0
    assert oracle.scale(oracle.SCALE_L2, 4.0, 9.0) == 0.25
    assert oracle.scale(oracle.SCALE_NONE, 4.0, 9.0) == 1.0


def test_eta_hat_geometric():
    rho, m, k, C = 0.7, 60, 25, 1.0
    delta = _geometric(rho, m)
    eps64 = 2.0 ** -53
    w = np.empty(m + 1)
    w[0] = (5 + 2 * C)
    w[1:] = ((3 + C) / rho + (2 + C)) * rho ** np.arange(1, m + 1)
    closed = eps64 * w[: k + 1].sum() + EPS32 * w[k:].sum()
    assert oracle.eta_hat(delta, k, m, C) == pytest.approx(closed, rel=1e-12)
