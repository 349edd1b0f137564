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
