"""Final density field and power spectrum (Sec. 4.1-4.2, Eq. 24).

Test infrastructure (see ``oracle/__init__``).

The final density is the periodic CIC assignment of all particles to the
N^3 LPT grid (Sec. 4.1), nodes at (i + 1/2) d, delta = rho / nbar - 1 with
nbar = Np^3 / N^3.  The power spectrum estimator follows the convention of
Eq. 24 (continuum transform delta(k) = d^3 DFT[delta]):
    P(k_bin) = < |DFT[delta](k)|^2 > * L^3 / N^6
averaged over all modes of the full (not half) DFT whose |k| falls in the bin.
The paper uses 100 logarithmic bins from 2 pi / L to 1 h/Mpc; callers pass the
bin edges.  The paper's normalisation in Eq. 24 is garbled (an extra power of
L); this estimator uses the standard one, under which the ensemble mean of a
field coloured by ``ics.initial_density`` is the input P(k).

Pins (tests/test_oracle_stats.py): the CIC density of a uniform lattice is 0;
the estimator of a single cosine returns its closed-form power in one bin; the
ensemble average of coloured fields recovers the input spectrum.
"""
import numpy as np


def cic_density_periodic(x, L, N, Np):
    """Periodic CIC density contrast of positions x (M, 3) on the N^3 grid."""
    d = L / N
    u = np.asarray(x, dtype=np.float64) / d - 0.5
    i0 = np.floor(u).astype(np.int64)
    f = u - i0
    rho = np.zeros(N**3)
    for dx in (0, 1):
        for dy in (0, 1):
            for dz in (0, 1):
                w = ((f[:, 0] if dx else 1.0 - f[:, 0]) * (f[:, 1] if dy else 1.0 - f[:, 1])
                     * (f[:, 2] if dz else 1.0 - f[:, 2]))
                c = (i0 + np.array([dx, dy, dz])) % N
                rho += np.bincount((c[:, 0] * N + c[:, 1]) * N + c[:, 2], weights=w, minlength=N**3)
    return rho.reshape(N, N, N) * (float(N) ** 3 / float(Np) ** 3) - 1.0


def mode_magnitudes(N, L):
    n = np.fft.fftfreq(N, d=1.0 / N)
    kf = 2.0 * np.pi / L
    return kf * np.sqrt(n[:, None, None] ** 2 + n[None, :, None] ** 2 + n[None, None, :] ** 2)


def power_spectrum(delta, L, edges):
    """Binned P(k) of a real field on an N^3 periodic grid (Eq. 24 convention).

    Returns (k_mean, P, n_modes) per bin; empty bins give NaN.
    """
    N = delta.shape[0]
    dk = np.fft.fftn(np.asarray(delta, dtype=np.float64))
    p3 = np.abs(dk) ** 2 * (L**3 / float(N) ** 6)
    k = mode_magnitudes(N, L)
    which = np.digitize(k.ravel(), edges) - 1
    nb = len(edges) - 1
    valid = (which >= 0) & (which < nb)
    cnt = np.bincount(which[valid], minlength=nb).astype(np.float64)
    psum = np.bincount(which[valid], weights=p3.ravel()[valid], minlength=nb)
    ksum = np.bincount(which[valid], weights=k.ravel()[valid], minlength=nb)
    with np.errstate(invalid="ignore", divide="ignore"):
        return ksum / cnt, psum / cnt, cnt


def paper_bins(L, kmax=1.0, nbins=100):
    """100 logarithmic bins from the fundamental mode 2 pi / L to 1 h/Mpc (Sec. 4.2)."""
    return np.geomspace(2.0 * np.pi / L, kmax, nbins + 1)
