"""Pins of the oracle's initial conditions (Sec. 3.1 A.1) against closed forms and statistics."""
import numpy as np

import synth_inputs
from oracle import ics, stats

COS = {k: synth_inputs.COSMOLOGY[k] for k in ("Om", "h", "ns", "sigma8")}


def test_single_mode_is_coloured_by_sqrt_power():
    # w = cos(k.x) has DFT N^3/2 at +-k; colouring multiplies by sqrt(P(|k|)/d^3) (A.1).
    N, L = 16, 100.0
    d = L / N
    x = np.arange(N)
    m = np.array([1, 2, 3])
    phase = 2 * np.pi * (m[0] * x[:, None, None] + m[1] * x[None, :, None] + m[2] * x[None, None, :]) / N
    w = np.cos(phase)
    delta = ics.initial_density(w, L, **COS)
    kmag = 2 * np.pi / L * np.sqrt((m**2).sum())
    pk = ics.power_spectrum_fn(COS["Om"], COS["h"], COS["ns"], COS["sigma8"])
    np.testing.assert_allclose(delta, np.sqrt(pk(kmag) / d**3) * w, rtol=1e-12, atol=1e-14)


def test_bbks_limits():
    # T -> 1 on large scales; T decreases monotonically; T ~ ln(q)/q^2 at large q.
    Om, h = COS["Om"], COS["h"]
    assert abs(ics.bbks_transfer(1e-9, Om, h) - 1.0) < 1e-6
    k = np.geomspace(1e-4, 1e2, 200)
    t = ics.bbks_transfer(k, Om, h)
    assert np.all(np.diff(t) < 0)
    q = 1e4
    big = ics.bbks_transfer(q * Om * h, Om, h)
    asym = np.log(2.34 * q) / (2.34 * q) / (6.71 * q)
    assert abs(big / asym - 1) < 0.05


def test_sigma8_normalisation_independent_quadrature():
    pk = ics.power_spectrum_fn(COS["Om"], COS["h"], COS["ns"], COS["sigma8"])
    lnk = np.linspace(np.log(1e-5), np.log(1e3), 400001)
    k = np.exp(lnk)
    integrand = k**3 * pk(k) * ics.tophat_window(8.0 * k) ** 2 / (2 * np.pi**2)
    s2 = np.trapezoid(integrand, lnk)
    assert abs(np.sqrt(s2) / COS["sigma8"] - 1) < 1e-6


def test_ensemble_power_matches_input_within_cosmic_variance():
    N, L = 16, 200.0
    edges = np.linspace(2 * np.pi / L * 0.5, np.pi * N / L, 7)
    pk = ics.power_spectrum_fn(COS["Om"], COS["h"], COS["ns"], COS["sigma8"])
    acc = []
    for seed in range(40):
        w = synth_inputs.white_noise(N, 1000 + seed)
        acc.append(stats.power_spectrum(ics.initial_density(w, L, **COS), L, edges)[1])
    meas = np.mean(acc, axis=0)
    # mode-averaged model in each bin
    kk = stats.mode_magnitudes(N, L)
    which = np.digitize(kk.ravel(), edges) - 1
    model = np.array([pk(kk.ravel()[(which == b) & (kk.ravel() > 0)]).mean() for b in range(len(edges) - 1)])
    _, _, nmodes = stats.power_spectrum(np.zeros((N, N, N)), L, edges)
    sigma = model * np.sqrt(2.0 / (nmodes * 40))   # each real mode appears twice in the full DFT
    assert np.all(np.abs(meas - model) < 5 * sigma)


def _bbks_taylor_from_publication():
    """Taylor coefficients t0..t4 of T(q) about q = 0, derived by hand from Bardeen, Bond,
    Kaiser and Szalay (1986, ApJ 304, 15, Eq. G3):
        T(q) = ln(1 + a q)/(a q) [1 + b q + (c q)^2 + (d q)^3 + (e q)^4]^(-1/4)
    with the constants as printed there, a = 2.34, b = 3.89, c = 16.1, d = 5.46, e = 6.71.
    ln(1 + a q)/(a q) = sum_n (-a q)^n / (n + 1); (1 + u)^(-1/4) = 1 - u/4 + 5u^2/32
    - 15u^3/128 + 195u^4/2048 - ...; the product is collected by powers of q.  Each constant
    enters a different order: a and b the first, c the second, d the third, e the fourth."""
    a, b, c, d, e = 2.34, 3.89, 16.1, 5.46, 6.71
    A = [1.0, -a / 2, a**2 / 3, -a**3 / 4, a**4 / 5]
    B = [1.0,
         -b / 4,
         -c**2 / 4 + 5 * b**2 / 32,
         -d**3 / 4 + (5 / 32) * 2 * b * c**2 - (15 / 128) * b**3,
         -e**4 / 4 + (5 / 32) * (c**4 + 2 * b * d**3) - (15 / 128) * 3 * b**2 * c**2 + (195 / 2048) * b**4]
    return [sum(A[i] * B[n - i] for i in range(n + 1)) for n in range(5)]


def test_bbks_taylor_coefficients_match_published_constants():
    # The oracle's T(q), sampled at Chebyshev nodes of [0, 0.01] and fitted, gives its own
    # Taylor coefficients; they must equal those of the published formula.  A 5 % change of
    # any one of the five constants moves some coefficient by more than 1 %.
    from numpy.polynomial import chebyshev as C, polynomial as Pn
    Om, h = COS["Om"], COS["h"]
    r, m = 0.01, 200
    x = np.cos(np.pi * (np.arange(m) + 0.5) / m)
    q = (x + 1) / 2 * r
    T = ics.bbks_transfer(q * Om * h, Om, h)
    series = Pn.Polynomial(C.cheb2poly(C.chebfit(x, T, 12)))(Pn.Polynomial([-1.0, 2.0 / r])).coef
    expect = _bbks_taylor_from_publication()
    assert abs(series[0] - 1.0) < 1e-13
    for n, tol in ((1, 1e-9), (2, 1e-8), (3, 1e-6), (4, 1e-4)):
        assert abs(series[n] / expect[n] - 1.0) < tol, (n, series[n], expect[n])


def test_bbks_close_to_eisenstein_hu_zero_baryon_fit():
    # Independent physics: the Eisenstein & Hu (1998, ApJ 496, 605, Eqs. 28-29) zero-baryon
    # transfer function, T0(q) = L0 / (L0 + C0 q^2), L0 = ln(2e + 1.8 q),
    # C0 = 14.2 + 731 / (1 + 62.5 q), q = k Theta^2 / Gamma (k in h/Mpc, Theta = 2.728/2.7),
    # fits the same CDM transfer function; the two fits agree within 7 % for
    # 0.01 <= k <= 1 h/Mpc at Gamma = Om h = 0.21 (measured: -0.4 % ... +6.1 %).
    Om, h = COS["Om"], COS["h"]
    k = np.geomspace(0.01, 1.0, 200)
    theta2 = (2.728 / 2.7) ** 2
    qe = k * theta2 / (Om * h)
    L0 = np.log(2 * np.e + 1.8 * qe)
    T_eh = L0 / (L0 + (14.2 + 731.0 / (1 + 62.5 * qe)) * qe**2)
    ratio = ics.bbks_transfer(k, Om, h) / T_eh
    assert np.all(np.abs(ratio - 1) < 0.07)
    assert np.all(ratio > 0.99)
