"""Background cosmology, growth factors and COLA time coefficients (FP64).

Test infrastructure (see ``oracle/__init__``).

Conventions (App. A of the paper): time variable a, H0 = 1, so the conformal
Hubble factor is  calH(a) = a H(a) = sqrt(Om/a + Ok + OL a^2)  with
Ok = 1 - Om - OL.  The drift prefactor is  calD(a) = 1/(a^2 calH)  (Eq. 37) and
the kick prefactor is  calK(a) = -(3/2) Om / (a calH)  (Eq. 38).

Growth factors.  D1 and D2 solve the linear and second-order growth equations
whose COLA operator identities are  V[D1] = D1  and  V[D2] = D2 - D1^2
(Eqs. 44-45).  Written with primes = d/dln a:
    D'' + (2 + dlnH/dlna) D' - (3/2) Om(a) D = 0                       (D1)
    D'' + (2 + dlnH/dlna) D' - (3/2) Om(a) D = -(3/2) Om(a) D1^2        (D2)
with the growing modes D1 -> a, D2 -> -(3/7) a^2 at early times, integrated
with fixed-step classical RK4 in ln a and normalised to D1(a=1) = 1 (the paper
normalises D1 at the initial conditions, Eq. 23; only the product D1 phi1
enters, so the normalisation point is a convention fixed once for both the
potentials and D1).

Time coefficients.  Modified discretisation of App. B with u(a) = a^nLPT,
t(a) = a (Eq. 60):
    alpha~(ai, af, aK) = aK^-nLPT  * int_ai^af a^(nLPT-2)/calH(a) da
    beta~(ai, af, aD)  = -(3/2) Om (af^nLPT - ai^nLPT) / (nLPT aD^nLPT calH(aD))
The integral uses adaptive Simpson quadrature written out below.  Standard
discretisation (App. B, the alternative the paper describes before adopting the
modified one): alpha_p = int_ai^af da/(a^2 calH), beta_delta = -(3/2) Om int da/(a calH).

KDK schedule (Eq. 52, read with the product running over the n-1 inner steps
so that no drift is applied twice; half-step times are arithmetic means in a):
    K(a0 -> a_1/2; F at a0),
    for k = 0..n-1:  D(a_k -> a_k+1; p at a_k+1/2),
                     K(a_k+1/2 -> a_k+3/2, or a_n at the last step; F at a_k+1)
so n drift steps use n+1 force evaluations.

Pins (tests/test_oracle_cosmology.py): Einstein-de Sitter closed forms for D1,
D2, alpha~ and beta~; the Heath integral for the LCDM linear growth factor;
finite-difference checks of V[D1] = D1 and V[D2] = D2 - D1^2; beta~ against its
defining integral; convergence of the KDK integrator to the exact linear-growth
trajectory.
"""
import numpy as np


def conformal_hubble(a, Om, OL):
    """calH(a) = a H(a) with H0 = 1 (App. A, below Eq. 38)."""
    a = np.asarray(a, dtype=np.float64)
    Ok = 1.0 - Om - OL
    return np.sqrt(Om / a + Ok + OL * a * a)


def drift_prefactor(a, Om, OL):
    """calD(a) = 1/(a^2 calH(a))  (Eq. 37)."""
    return 1.0 / (a * a * conformal_hubble(a, Om, OL))


def kick_prefactor(a, Om, OL):
    """calK(a) = -(3/2) Om / (a calH(a))  (Eq. 38, H0 = 1)."""
    return -1.5 * Om / (a * conformal_hubble(a, Om, OL))


def _growth_rhs(y, S, Om, OL):
    """Right-hand side of the growth equations in y = ln a.

    S has rows (D1, D1', D2, D2'), primes = d/dln a.
    """
    Ok = 1.0 - Om - OL
    a = np.exp(y)
    E2 = Om / a**3 + Ok / a**2 + OL
    dlnH = (-3.0 * Om / a**3 - 2.0 * Ok / a**2) / (2.0 * E2)
    Om_a = (Om / a**3) / E2
    D1, D1p, D2, D2p = S
    return np.array([
        D1p,
        -(2.0 + dlnH) * D1p + 1.5 * Om_a * D1,
        D2p,
        -(2.0 + dlnH) * D2p + 1.5 * Om_a * (D2 - D1 * D1),
    ])


def growth_factors(a, Om, OL, a_start=1e-6, nsteps=5000):
    """D1, D2 and their derivatives dD/da at the scale factors ``a``.

    Returns a dict of arrays (same shape as ``a``): D1, D2, dD1da, dD2da,
    normalised so that D1(1) = 1 (D2 scaled by the square of the same factor,
    since the D2 equation is quadratic in D1).

    Every requested a (plus a = 1) is integrated from a_start with its own
    uniform RK4 step in ln a, all in one vectorised sweep.
    """
    a = np.atleast_1d(np.asarray(a, dtype=np.float64))
    targets = np.concatenate([a.ravel(), [1.0]])
    y0 = np.log(a_start)
    h = (np.log(targets) - y0) / nsteps
    S = np.array([
        np.full_like(targets, a_start),
        np.full_like(targets, a_start),
        np.full_like(targets, -3.0 / 7.0 * a_start**2),
        np.full_like(targets, -6.0 / 7.0 * a_start**2),
    ])
    y = np.full_like(targets, y0)
    for _ in range(nsteps):
        k1 = _growth_rhs(y, S, Om, OL)
        k2 = _growth_rhs(y + 0.5 * h, S + 0.5 * h * k1, Om, OL)
        k3 = _growth_rhs(y + 0.5 * h, S + 0.5 * h * k2, Om, OL)
        k4 = _growth_rhs(y + h, S + h * k3, Om, OL)
        S = S + (h / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
        y = y + h
    norm = S[0, -1]
    D1 = S[0, :-1] / norm
    D2 = S[2, :-1] / norm**2
    dD1da = S[1, :-1] / norm / targets[:-1]
    dD2da = S[3, :-1] / norm**2 / targets[:-1]
    shape = np.shape(a)
    return {
        "D1": D1.reshape(shape), "D2": D2.reshape(shape),
        "dD1da": dD1da.reshape(shape), "dD2da": dD2da.reshape(shape),
    }


def adaptive_simpson(f, lo, hi, rtol=1e-14, max_depth=60):
    """Adaptive Simpson quadrature of a smooth scalar function on [lo, hi]."""
    def simpson(a, fa, b, fb):
        m = 0.5 * (a + b)
        fm = f(m)
        return m, fm, (b - a) / 6.0 * (fa + 4.0 * fm + fb)

    def recurse(a, fa, b, fb, m, fm, whole, tol, depth):
        lm, flm, left = simpson(a, fa, m, fm)
        rm, frm, right = simpson(m, fm, b, fb)
        delta = left + right - whole
        if depth <= 0 or abs(delta) <= 15.0 * tol:
            return left + right + delta / 15.0
        return (recurse(a, fa, m, fm, lm, flm, left, 0.5 * tol, depth - 1)
                + recurse(m, fm, b, fb, rm, frm, right, 0.5 * tol, depth - 1))

    if hi == lo:
        return 0.0
    flo, fhi = f(lo), f(hi)
    m, fm, whole = simpson(lo, flo, hi, fhi)
    tol = rtol * max(abs(whole), 1e-300)
    return recurse(lo, flo, hi, fhi, m, fm, whole, tol, max_depth)


def alpha_tilde(ai, af, aK, Om, OL, nLPT=-2.5):
    """Modified drift coefficient alpha~_p(ai, af, aK) (Eq. 60, first part)."""
    integrand = lambda x: x ** (nLPT - 2.0) / float(conformal_hubble(x, Om, OL))
    return aK ** (-nLPT) * adaptive_simpson(integrand, ai, af)


def beta_tilde(ai, af, aD, Om, OL, nLPT=-2.5):
    """Modified kick coefficient beta~_delta(ai, af, aD) (Eq. 60, second part)."""
    return (-1.5 * Om * (af ** nLPT - ai ** nLPT)
            / (nLPT * aD ** nLPT * float(conformal_hubble(aD, Om, OL))))


def alpha_standard(ai, af, Om, OL):
    """Standard drift factor (App. B, Eq. 50 with t = a): int_ai^af da / (a^2 calH(a))."""
    return adaptive_simpson(lambda x: float(drift_prefactor(x, Om, OL)), ai, af)


def beta_standard(ai, af, Om, OL):
    """Standard kick factor (App. B, Eq. 50 with t = a): -(3/2) Om int_ai^af da / (a calH(a))."""
    return adaptive_simpson(lambda x: float(kick_prefactor(x, Om, OL)), ai, af)


def kdk_schedule(a_i, a_f, nsteps, Om, OL, nLPT=-2.5, stepping="modified"):
    """Coefficients of the KDK sequence (Eq. 52 with the COLA operators Eqs. 53-54).

    stepping: "modified" (u(a) = a^nLPT factors, the paper's choice) or "standard"
    (the time integrals of the drift and kick prefactors over each interval, App. B).

    Time steps are linear in a.  Returns a dict with, for each of the
    nsteps + 1 force evaluations k (force at a_k):
      a_force[k], D1[k], D2[k]   growth factors at the force time
      beta[k]                    kick coefficient of the kick that uses this force
      kick_from[k], kick_to[k]   kick interval
    and for each of the nsteps drifts k (a_k -> a_k+1, momentum at a_k+1/2):
      alpha[k], dD1[k], dD2[k]   drift coefficient and growth increments
    plus the L+/L- data at a_i and a_f (D1, D2, dD1da, dD2da).
    """
    n = int(nsteps)
    a = a_i + (a_f - a_i) * np.arange(n + 1, dtype=np.float64) / n
    ah = 0.5 * (a[:-1] + a[1:])
    g = growth_factors(np.concatenate([a, [a_i, a_f]]), Om, OL)
    D1 = g["D1"][: n + 1]
    D2 = g["D2"][: n + 1]
    kick_from = np.empty(n + 1)
    kick_to = np.empty(n + 1)
    beta = np.empty(n + 1)
    for k in range(n + 1):
        kick_from[k] = a[0] if k == 0 else ah[k - 1]
        kick_to[k] = ah[k] if k < n else a[n]
        if stepping == "standard":
            beta[k] = beta_standard(kick_from[k], kick_to[k], Om, OL)
        else:
            beta[k] = beta_tilde(kick_from[k], kick_to[k], a[k], Om, OL, nLPT)
    if stepping == "standard":
        alpha = np.array([alpha_standard(a[k], a[k + 1], Om, OL) for k in range(n)])
    else:
        alpha = np.array([alpha_tilde(a[k], a[k + 1], ah[k], Om, OL, nLPT) for k in range(n)])
    dD1 = D1[1:] - D1[:-1]
    dD2 = D2[1:] - D2[:-1]
    return {
        "a": a, "a_half": ah, "a_force": a.copy(), "D1": D1, "D2": D2,
        "beta": beta, "kick_from": kick_from, "kick_to": kick_to,
        "alpha": alpha, "dD1": dD1, "dD2": dD2,
        "D1_i": g["D1"][n + 1], "D2_i": g["D2"][n + 1],
        "D1_f": g["D1"][n + 2], "D2_f": g["D2"][n + 2],
        "dD1da_f": g["dD1da"][n + 2], "dD2da_f": g["dD2da"][n + 2],
        "dD1da_i": g["dD1da"][n + 1], "dD2da_i": g["dD2da"][n + 1],
    }
