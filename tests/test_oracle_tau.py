"""Pins of the smoothing rules of §3.6 (oracle.mlmc.tau_exponential, tau_matern).

The paper leaves the constant ratio C_s / C_alpha to the user, so these tests
take it as a free input and check what the paper fixes for every value of it:

* the exponential rule (§3.6, no padding, s = 4 h^-2) is the tau at which the
  two terms of the bound of the exponential-covariance corollary are equal,
  C_alpha h^alpha = C_s (s - tau + 1)^-1 tau;
* the Matern rule comes from the Matern corollary's bound
  C_s s^-1/2 h^-1 (s - tau + 1)^-(1+nu)/2 tau balanced against C_alpha h^alpha,
  with s = 4 (1/h + J)^2 under smooth periodisation;
* at nu = 1 and J = 0 the Matern bound is half the exponential one
  (s^-1/2 h^-1 = 1/2 when s = 4 h^-2), so the bisection of the Matern rule
  must return the exponential closed form with C_s / C_alpha halved. The two
  rules are separate code (closed form and bisection), so a dropped factor,
  a wrong exponent or a misplaced J in either fails here.
"""
import math

import pytest

from oracle import mlmc

ALPHAS = (0.5, 1.0, 1.5, 2.0)
RATIOS = (0.05, 1.0, 20.0)          # C_s / C_alpha
HS = (1 / 8, 1 / 32, 1 / 128)


@pytest.mark.parametrize("alpha", ALPHAS)
@pytest.mark.parametrize("ratio", RATIOS)
@pytest.mark.parametrize("h", HS)
def test_exponential_rule_balances_the_bound(alpha, ratio, h):
    s = 4.0 / (h * h)
    tau = mlmc.tau_exponential(s, alpha, ratio)
    c_alpha, c_s = 1.0, ratio
    discretisation = c_alpha * h ** alpha
    smoothing = c_s * tau / (s - tau + 1.0)
    assert math.isclose(discretisation, smoothing, rel_tol=1e-12)


@pytest.mark.parametrize("alpha", ALPHAS)
@pytest.mark.parametrize("ratio", RATIOS)
@pytest.mark.parametrize("h", HS)
@pytest.mark.parametrize("J", (0, 8, 32))
@pytest.mark.parametrize("nu", (0.5, 1.5))
def test_matern_rule_balances_the_bound(alpha, ratio, h, J, nu):
    s = 4.0 * (1.0 / h + J) ** 2
    tau = mlmc.tau_matern(h, J, nu, alpha, ratio)
    if tau in (1.0, s):
        pytest.skip("balance point outside [1, s]: the rule clamps")
    c_alpha, c_s = 1.0, ratio
    discretisation = c_alpha * h ** alpha
    smoothing = c_s / math.sqrt(s) / h * (s - tau + 1.0) ** (-0.5 * (1.0 + nu)) * tau
    assert math.isclose(discretisation, smoothing, rel_tol=1e-9)


@pytest.mark.parametrize("alpha", ALPHAS)
@pytest.mark.parametrize("ratio", RATIOS)
@pytest.mark.parametrize("h", HS)
def test_matern_rule_at_nu_one_is_the_exponential_rule(alpha, ratio, h):
    s = 4.0 / (h * h)
    t_m = mlmc.tau_matern(h, 0, 1.0, alpha, ratio)
    t_e = mlmc.tau_exponential(s, alpha, ratio / 2.0)
    # the closed form is not restricted to [1, s] (at alpha = 2 and a large
    # C_s / C_alpha it falls below 1); the bisection clamps to that interval
    assert math.isclose(t_m, min(max(t_e, 1.0), s), rel_tol=1e-9)


def test_more_weight_on_smoothing_drops_fewer_eigenvalues():
    """A larger C_s / C_alpha (a costlier smoothing error) lowers tau in both
    rules: the exponential closed form decreases in it, and the Matern
    equation's left side increases in tau while its right side falls."""
    for alpha in ALPHAS:
        taus = [mlmc.tau_exponential(4096.0, alpha, r) for r in (0.1, 1.0, 10.0)]
        assert taus[0] > taus[1] > taus[2]
        taus = [mlmc.tau_matern(1 / 32, 4, 1.5, alpha, r) for r in (0.1, 1.0, 10.0)]
        assert taus[0] > taus[1] > taus[2]
