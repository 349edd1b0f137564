"""Pins of the oracle's cosmology and time integration (App. A-B) against closed forms."""
import numpy as np
import pytest
from scipy import integrate

from oracle import cosmology, scola


A_TEST = np.array([0.02, 0.05, 0.1, 0.3, 0.6, 1.0])


def test_eds_growth_closed_form():
    # Einstein-de Sitter: D1 = a, D2 = -(3/7) a^2 exactly (growing modes of Eqs. 44-45).
    g = cosmology.growth_factors(A_TEST, 1.0, 0.0)
    np.testing.assert_allclose(g["D1"], A_TEST, rtol=1e-10)
    np.testing.assert_allclose(g["D2"], -3.0 / 7.0 * A_TEST**2, rtol=1e-10)
    np.testing.assert_allclose(g["dD1da"], np.ones_like(A_TEST), rtol=1e-10)
    np.testing.assert_allclose(g["dD2da"], -6.0 / 7.0 * A_TEST, rtol=1e-10)


def test_lcdm_growth_matches_heath_integral():
    # Matter + Lambda: D1(a) proportional to H(a) int_0^a da' / (a' H(a'))^3.
    Om, OL = 0.3, 0.7
    H = lambda a: np.sqrt(Om / a**3 + OL)
    heath = lambda a: H(a) * integrate.quad(lambda x: 1.0 / (x * H(x)) ** 3, 0.0, a,
                                            epsabs=0, epsrel=1e-13, limit=200)[0]
    ref = np.array([heath(a) for a in A_TEST]) / heath(1.0)
    g = cosmology.growth_factors(A_TEST, Om, OL)
    np.testing.assert_allclose(g["D1"], ref, rtol=1e-9)
    # and the LCDM D2 is close to the Bouchet et al. fit -3/7 D1^2 Om(a)^(-1/143)
    Om_a = Om / A_TEST**3 / H(A_TEST) ** 2
    np.testing.assert_allclose(g["D2"], -3.0 / 7.0 * g["D1"] ** 2 * Om_a ** (-1.0 / 143.0), rtol=2e-3)


@pytest.mark.parametrize("Om,OL", [(0.3, 0.7), (1.0, 0.0), (0.25, 0.6)])
def test_cola_operator_identities(Om, OL):
    # V[f](a) = -(1/calK) d/da (a^2 calH df/da);  V[D1] = D1, V[D2] = D2 - D1^2 (Eqs. 44-45).
    a = np.array([0.05, 0.2, 0.5, 0.9])
    h = 1e-4 * a
    gp = cosmology.growth_factors(a + h, Om, OL)
    gm = cosmology.growth_factors(a - h, Om, OL)
    g0 = cosmology.growth_factors(a, Om, OL)
    w = lambda aa, gg, key: aa**2 * cosmology.conformal_hubble(aa, Om, OL) * gg[key]
    K = cosmology.kick_prefactor(a, Om, OL)
    V1 = -(w(a + h, gp, "dD1da") - w(a - h, gm, "dD1da")) / (2 * h) / K
    V2 = -(w(a + h, gp, "dD2da") - w(a - h, gm, "dD2da")) / (2 * h) / K
    np.testing.assert_allclose(V1, g0["D1"], rtol=1e-6)
    np.testing.assert_allclose(V2, g0["D2"] - g0["D1"] ** 2, rtol=1e-6)


def test_alpha_tilde_eds_closed_form():
    # EdS, n_LPT = -2.5: alpha~ = aK^2.5 (ai^-3 - af^-3) / 3  (Eq. 60 integrated by hand).
    for ai, af, aK in [(0.02, 0.118, 0.069), (0.5, 0.55, 0.525), (0.9, 1.0, 0.95)]:
        exact = aK**2.5 * (ai**-3 - af**-3) / 3.0
        assert abs(cosmology.alpha_tilde(ai, af, aK, 1.0, 0.0) / exact - 1) < 1e-12


def test_beta_tilde_against_definition():
    # beta~ = (u(af) - u(ai)) calK(aD) / u'(aD) with u = a^nLPT (Eq. 59); u' by finite difference.
    n = -2.5
    for (Om, OL) in [(0.3, 0.7), (1.0, 0.0)]:
        for ai, af, aD in [(0.02, 0.069, 0.02), (0.4, 0.5, 0.45), (0.95, 1.0, 1.0)]:
            hh = 1e-5 * aD
            du = ((aD + hh) ** n - (aD - hh) ** n) / (2 * hh)
            ref = (af**n - ai**n) * cosmology.kick_prefactor(aD, Om, OL) / du
            assert abs(cosmology.beta_tilde(ai, af, aD, Om, OL, n) / ref - 1) < 1e-8


def test_modified_coefficients_reduce_to_standard_on_short_steps():
    # Over a short step the modified factors approach the standard alpha_p, beta_delta (Eq. 51).
    Om, OL = 0.3, 0.7
    ai, af = 0.5, 0.5005
    am = 0.5 * (ai + af)
    std_alpha = integrate.quad(lambda a: cosmology.drift_prefactor(a, Om, OL), ai, af, epsrel=1e-13)[0]
    std_beta = integrate.quad(lambda a: cosmology.kick_prefactor(a, Om, OL), ai, af, epsrel=1e-13)[0]
    assert abs(cosmology.alpha_tilde(ai, af, am, Om, OL) / std_alpha - 1) < 1e-6
    assert abs(cosmology.beta_tilde(ai, af, am, Om, OL) / std_beta - 1) < 1e-6


def test_kdk_converges_to_linear_growth_trajectory():
    # With Psi1 = Psi2 = 0 (trivial LPT frame) and the force F(a) = D1(a) G, the exact
    # solution of Eqs. 46-47 is s = -D1(a) G, p = -a^2 calH dD1/da G (from V[D1] = D1).
    # The KDK sequence must converge to it at second order.
    Om, OL, ai, af = 0.3, 0.7, 0.02, 1.0
    G = np.array([[1.0, -2.0, 0.5]])
    zero = np.zeros_like(G)
    errs = []
    for n in (40, 80, 160):
        sched = cosmology.kdk_schedule(ai, af, n, Om, OL)
        s0 = -sched["D1_i"] * G
        p0 = -ai**2 * cosmology.conformal_hubble(ai, Om, OL) * sched["dD1da_i"] * G
        s, p, _ = scola.kdk_integrate(s0, p0, zero, zero, sched,
                                      lambda k, s: (sched["D1"][k] * G, None))
        s_exact = -sched["D1_f"] * G
        p_exact = -af**2 * cosmology.conformal_hubble(af, Om, OL) * sched["dD1da_f"] * G
        errs.append(max(np.abs(s - s_exact).max() / np.abs(s_exact).max(),
                        np.abs(p - p_exact).max() / np.abs(p_exact).max()))
    # steps are linear in a from a_i = 0.02, so the first step is large; the
    # error still falls by ~4x per halving (second order)
    assert errs[2] < 5e-3
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5


def test_schedule_structure():
    sched = cosmology.kdk_schedule(0.02, 1.0, 10, 0.3, 0.7)
    assert len(sched["beta"]) == 11 and len(sched["alpha"]) == 10
    assert sched["kick_from"][0] == 0.02 and sched["kick_to"][-1] == 1.0
    np.testing.assert_allclose(sched["kick_to"][:-1], sched["kick_from"][1:])
    assert np.all(sched["beta"] < 0) and np.all(sched["alpha"] > 0)


def test_standard_factors_edS_closed_form():
    # Standard discretisation (App. B): alpha_p = int da / (a^2 calH), beta_delta =
    # -(3/2) Om int da / (a calH).  In EdS (Om = 1, calH = a^-1/2) these are
    # 2 (ai^-1/2 - af^-1/2) and -3 (af^1/2 - ai^1/2).
    for ai, af in [(0.02, 0.069), (0.3, 0.35), (0.9, 1.0)]:
        assert abs(cosmology.alpha_standard(ai, af, 1.0, 0.0) / (2 * (ai**-0.5 - af**-0.5)) - 1) < 1e-12
        assert abs(cosmology.beta_standard(ai, af, 1.0, 0.0) / (-3 * (af**0.5 - ai**0.5)) - 1) < 1e-12


def test_standard_schedule_uses_interval_integrals():
    sched = cosmology.kdk_schedule(0.02, 1.0, 10, 0.3, 0.7, stepping="standard")
    for k in range(10):
        assert sched["alpha"][k] == cosmology.alpha_standard(sched["a"][k], sched["a"][k + 1], 0.3, 0.7)
    for k in range(11):
        assert sched["beta"][k] == cosmology.beta_standard(sched["kick_from"][k], sched["kick_to"][k], 0.3, 0.7)
    # the modified factors differ on these long steps (not the same scheme by mistake)
    mod = cosmology.kdk_schedule(0.02, 1.0, 10, 0.3, 0.7)
    assert abs(mod["alpha"][0] / sched["alpha"][0] - 1) > 1e-3


def test_standard_kdk_converges_to_linear_growth_trajectory():
    # The same exact trajectory as above (trivial LPT frame, F = D1(a) G) with the standard
    # factors: second-order convergence.
    Om, OL, ai, af = 0.3, 0.7, 0.02, 1.0
    G = np.array([[1.0, -2.0, 0.5]])
    zero = np.zeros_like(G)
    errs = []
    for n in (40, 80, 160):
        sched = cosmology.kdk_schedule(ai, af, n, Om, OL, stepping="standard")
        s0 = -sched["D1_i"] * G
        p0 = -ai**2 * cosmology.conformal_hubble(ai, Om, OL) * sched["dD1da_i"] * G
        s, p, _ = scola.kdk_integrate(s0, p0, zero, zero, sched, lambda k, s: (sched["D1"][k] * G, None))
        s_exact = -sched["D1_f"] * G
        p_exact = -af**2 * cosmology.conformal_hubble(af, Om, OL) * sched["dD1da_f"] * G
        errs.append(max(np.abs(s - s_exact).max() / np.abs(s_exact).max(),
                        np.abs(p - p_exact).max() / np.abs(p_exact).max()))
    assert errs[2] < 5e-3
    assert errs[0] / errs[1] > 3.5 and errs[1] / errs[2] > 3.5
