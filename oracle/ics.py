"""Initial density contrast by the convolution approach (Sec. 3.1, step A.1).

Test infrastructure (see ``oracle/__init__``).

The white-noise field w (unit variance per cell, an input) is coloured in
Fourier space:  DFT[delta](k) = DFT[w](k) * sqrt(P(|k|) / d^3),  d = L/N, with
the k = 0 mode set to zero, and delta = IDFT.  With <|DFT w|^2> = N^3 this gives
<|DFT delta|^2> = N^3 P / d^3, i.e. the continuum spectrum P(k) in the
convention of Eq. 24 (delta_cont(k) = d^3 DFT[delta]).

P(k) = A k^ns T_BBKS(k/Gamma)^2 with Gamma = Om h (k in h/Mpc) and the BBKS
transfer function.  A is fixed by sigma8 (top-hat radius 8 Mpc/h) at a = 1,
where D1 = 1.  The paper itself uses the Eisenstein-Hu fit (Sec. 4); the BBKS
form and the parameters are the workload's.

Pins (tests/test_oracle_ics.py): a single Fourier mode of w produces a cosine
of amplitude sqrt(P/d^3) (closed form); T(q -> 0) = 1; the Taylor coefficients of
T to fourth order in q equal those derived by hand from the published BBKS
constants (each of the five constants enters one order, so a 5 % error in any
of them fails); T stays within 7 % of the independent Eisenstein & Hu (1998)
zero-baryon fit for 0.01 <= k <= 1 h/Mpc; the sigma8 integral of the normalised
spectrum reproduces sigma8 with an independent quadrature; the ensemble P(k) of
coloured fields matches P within cosmic variance.
"""
import numpy as np
from scipy import integrate


def bbks_transfer(k, Om, h):
    """BBKS (1986) transfer function with shape parameter Gamma = Om h."""
    k = np.asarray(k, dtype=np.float64)
    q = k / (Om * h)
    with np.errstate(divide="ignore", invalid="ignore"):
        t = (np.log1p(2.34 * q) / (2.34 * q)
             * (1.0 + 3.89 * q + (16.1 * q) ** 2 + (5.46 * q) ** 3 + (6.71 * q) ** 4) ** -0.25)
    return np.where(q > 0, t, 1.0)


def tophat_window(x):
    """Fourier transform of a normalised spherical top hat, W(x) = 3 j1(x)/x."""
    x = np.asarray(x, dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        w = 3.0 * (np.sin(x) - x * np.cos(x)) / x**3
    return np.where(x > 1e-4, w, 1.0 - x * x / 10.0)


def sigma_r_squared(pk, R=8.0):
    """sigma_R^2 = int dk k^2 P(k) W^2(kR) / (2 pi^2), integrated in ln k."""
    f = lambda lnk: (np.exp(lnk) ** 3 * pk(np.exp(lnk)) * tophat_window(np.exp(lnk) * R) ** 2
                     / (2.0 * np.pi**2))
    val, _ = integrate.quad(f, np.log(1e-5), np.log(1e3), limit=1000, epsabs=0.0, epsrel=1e-12)
    return val


def power_spectrum_fn(Om, h, ns, sigma8):
    """Return P(k) (k in h/Mpc, P in (Mpc/h)^3) normalised to sigma8 at a = 1."""
    unnorm = lambda k: np.asarray(k, dtype=np.float64) ** ns * bbks_transfer(k, Om, h) ** 2
    A = sigma8**2 / sigma_r_squared(unnorm, 8.0)
    return lambda k: A * unnorm(k)


def fourier_wavenumbers(N, L):
    """Integer-wrapped wavenumbers 2 pi n / L for the rfftn layout (kx, ky, kz)."""
    n_full = np.fft.fftfreq(N, d=1.0 / N)
    n_half = np.fft.rfftfreq(N, d=1.0 / N)
    kf = 2.0 * np.pi / L
    kx = kf * n_full[:, None, None]
    ky = kf * n_full[None, :, None]
    kz = kf * n_half[None, None, :]
    return kx, ky, kz


def initial_density(w, L, Om, h, ns, sigma8):
    """delta_i on the N^3 LPT grid from white noise w (Sec. 3.1, A.1)."""
    w = np.asarray(w, dtype=np.float64)
    N = w.shape[0]
    d = L / N
    pk = power_spectrum_fn(Om, h, ns, sigma8)
    kx, ky, kz = fourier_wavenumbers(N, L)
    kmag = np.sqrt(kx**2 + ky**2 + kz**2)
    amp = np.zeros_like(kmag)
    nz = kmag > 0
    amp[nz] = np.sqrt(pk(kmag[nz]) / d**3)
    return np.fft.irfftn(np.fft.rfftn(w) * amp, s=w.shape, axes=(0, 1, 2))
