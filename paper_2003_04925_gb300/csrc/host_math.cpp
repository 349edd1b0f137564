// FP64 host mathematics: background, growth factors, COLA time coefficients,
// power-spectrum amplitude.
//
// calH(a) = a H(a) with H0 = 1:  calH^2 = Om/a + Ok + OL a^2   (App. A)
// D1, D2 solve the growth equations whose COLA identities are V[D1] = D1 and
// V[D2] = D2 - D1^2 (Eqs. 44-45); in y = ln a with primes d/dy:
//   D'' + (2 + dlnH/dy) D' = (3/2) Om(a) D              (D1)
//   D'' + (2 + dlnH/dy) D' = (3/2) Om(a) (D - D1^2)     (D2)
// integrated with an adaptive Dormand-Prince 5(4) pair from the growing modes
// D1 = a, D2 = -(3/7) a^2 at a = 1e-6, normalised to D1(1) = 1.
// Modified time stepping u(a) = a^nLPT (App. B, Eq. 60):
//   alpha~(ai, af, aK) = aK^-nLPT int_ai^af a^(nLPT-2) / calH da   (Gauss-Legendre)
//   beta~(ai, af, aD)  = -(3/2) Om (af^n - ai^n) / (n aD^n calH(aD))
// Standard time stepping (App. B): alpha_p = int da/(a^2 calH), beta = -(3/2) Om int da/(a calH).
// KDK sequence (Eq. 52, product over the n-1 inner steps, half steps at the
// arithmetic mean): K(a0->a1/2; F(a0)), then for k = 0..n-1
// D(ak->ak+1; p(ak+1/2)), K(ak+1/2 -> ak+3/2 or an; F(ak+1)).
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.h"

namespace scola {

double conformal_hubble(double a, double Om, double OL) {
    const double Ok = 1.0 - Om - OL;
    return std::sqrt(Om / a + Ok + OL * a * a);
}

namespace {

void growth_rhs(double y, const double *s, double Om, double OL, double *out) {
    const double Ok = 1.0 - Om - OL;
    const double a = std::exp(y);
    const double a2 = a * a, a3 = a2 * a;
    const double E2 = Om / a3 + Ok / a2 + OL;
    const double dlnH = (-3.0 * Om / a3 - 2.0 * Ok / a2) / (2.0 * E2);
    const double Oma = (Om / a3) / E2;
    out[0] = s[1];
    out[1] = -(2.0 + dlnH) * s[1] + 1.5 * Oma * s[0];
    out[2] = s[3];
    out[3] = -(2.0 + dlnH) * s[3] + 1.5 * Oma * (s[2] - s[0] * s[0]);
}

// One Dormand-Prince 5(4) step; returns the 5th-order solution and an error norm.
double dp45_step(double y, double h, const double *s, double Om, double OL, double *s5) {
    static const double c2 = 1.0 / 5, c3 = 3.0 / 10, c4 = 4.0 / 5, c5 = 8.0 / 9;
    static const double a21 = 1.0 / 5;
    static const double a31 = 3.0 / 40, a32 = 9.0 / 40;
    static const double a41 = 44.0 / 45, a42 = -56.0 / 15, a43 = 32.0 / 9;
    static const double a51 = 19372.0 / 6561, a52 = -25360.0 / 2187, a53 = 64448.0 / 6561,
                        a54 = -212.0 / 729;
    static const double a61 = 9017.0 / 3168, a62 = -355.0 / 33, a63 = 46732.0 / 5247,
                        a64 = 49.0 / 176, a65 = -5103.0 / 18656;
    static const double b1 = 35.0 / 384, b3 = 500.0 / 1113, b4 = 125.0 / 192,
                        b5 = -2187.0 / 6784, b6 = 11.0 / 84;
    static const double e1 = 5179.0 / 57600, e3 = 7571.0 / 16695, e4 = 393.0 / 640,
                        e5 = -92097.0 / 339200, e6 = 187.0 / 2100, e7 = 1.0 / 40;
    double k1[4], k2[4], k3[4], k4[4], k5[4], k6[4], k7[4], t[4];
    growth_rhs(y, s, Om, OL, k1);
    for (int i = 0; i < 4; ++i) t[i] = s[i] + h * a21 * k1[i];
    growth_rhs(y + c2 * h, t, Om, OL, k2);
    for (int i = 0; i < 4; ++i) t[i] = s[i] + h * (a31 * k1[i] + a32 * k2[i]);
    growth_rhs(y + c3 * h, t, Om, OL, k3);
    for (int i = 0; i < 4; ++i) t[i] = s[i] + h * (a41 * k1[i] + a42 * k2[i] + a43 * k3[i]);
    growth_rhs(y + c4 * h, t, Om, OL, k4);
    for (int i = 0; i < 4; ++i)
        t[i] = s[i] + h * (a51 * k1[i] + a52 * k2[i] + a53 * k3[i] + a54 * k4[i]);
    growth_rhs(y + c5 * h, t, Om, OL, k5);
    for (int i = 0; i < 4; ++i)
        t[i] = s[i] + h * (a61 * k1[i] + a62 * k2[i] + a63 * k3[i] + a64 * k4[i] + a65 * k5[i]);
    growth_rhs(y + h, t, Om, OL, k6);
    for (int i = 0; i < 4; ++i)
        s5[i] = s[i] + h * (b1 * k1[i] + b3 * k3[i] + b4 * k4[i] + b5 * k5[i] + b6 * k6[i]);
    growth_rhs(y + h, s5, Om, OL, k7);
    double err = 0.0;
    for (int i = 0; i < 4; ++i) {
        const double s4 = s[i] + h * (e1 * k1[i] + e3 * k3[i] + e4 * k4[i] + e5 * k5[i] +
                                      e6 * k6[i] + e7 * k7[i]);
        const double sc = 1e-300 + 1e-13 * std::max(std::fabs(s[i]), std::fabs(s5[i]));
        err = std::max(err, std::fabs(s5[i] - s4) / sc);
    }
    return err;
}

// Integrate the growth state from y0 to y1 adaptively.
void integrate_growth(double &y, double y1, double *s, double Om, double OL, double &h) {
    while (y < y1) {
        double step = std::min(h, y1 - y);
        double s5[4];
        const double err = dp45_step(y, step, s, Om, OL, s5);
        if (err <= 1.0) {
            y = (step == y1 - y) ? y1 : y + step;
            for (int i = 0; i < 4; ++i) s[i] = s5[i];
        }
        const double fac = err > 0 ? 0.9 * std::pow(err, -0.2) : 5.0;
        const double nh = step * std::min(5.0, std::max(0.2, fac));
        if (err <= 1.0 && step < h) {
            // last partial step to land on the target: keep the nominal step
            h = std::max(h, nh);
        } else {
            h = nh;
        }
    }
}

// Gauss-Legendre nodes and weights on [-1, 1] by Newton iteration on P_n.
void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < (n + 1) / 2; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
        for (int it = 0; it < 100; ++it) {
            double p1 = 1.0, p2 = 0.0;
            for (int j = 1; j <= n; ++j) {
                const double p3 = p2;
                p2 = p1;
                p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
            }
            const double dp = n * (z * p1 - p2) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        double p1 = 1.0, p2 = 0.0;
        for (int j = 1; j <= n; ++j) {
            const double p3 = p2;
            p2 = p1;
            p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
        }
        const double dp = n * (z * p1 - p2) / (z * z - 1.0);
        x[i] = -z;
        x[n - 1 - i] = z;
        w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

template <class F>
double composite_gl(F f, double lo, double hi, int panels, int order) {
    static std::vector<double> gx, gw;
    static int cached = 0;
    if (cached != order) {
        gauss_legendre(order, gx, gw);
        cached = order;
    }
    const double hp = (hi - lo) / panels;
    double sum = 0.0;
    for (int p = 0; p < panels; ++p) {
        const double mid = lo + (p + 0.5) * hp;
        double part = 0.0;
        for (int i = 0; i < order; ++i) part += gw[i] * f(mid + 0.5 * hp * gx[i]);
        sum += 0.5 * hp * part;
    }
    return sum;
}

double bbks_T(double k, double Om, double h) {
    const double q = k / (Om * h);
    if (q <= 0) return 1.0;
    const double poly = 1.0 + 3.89 * q + std::pow(16.1 * q, 2) + std::pow(5.46 * q, 3) +
                        std::pow(6.71 * q, 4);
    return std::log1p(2.34 * q) / (2.34 * q) * std::pow(poly, -0.25);
}

double tophat(double x) {
    if (x < 1e-4) return 1.0 - x * x / 10.0;
    return 3.0 * (std::sin(x) - x * std::cos(x)) / (x * x * x);
}

}  // namespace

double bbks_transfer(double k, double Om, double h) { return bbks_T(k, Om, h); }

void growth_factors(double Om, double OL, const std::vector<double> &a, std::vector<double> &D1,
                    std::vector<double> &D2, std::vector<double> &dD1da,
                    std::vector<double> &dD2da) {
    // targets = requested a plus a = 1 (normalisation), visited in increasing order
    std::vector<double> tg = a;
    tg.push_back(1.0);
    const size_t n = tg.size();
    std::vector<size_t> order(n);
    for (size_t i = 0; i < n; ++i) order[i] = i;
    std::sort(order.begin(), order.end(), [&](size_t x, size_t y) { return tg[x] < tg[y]; });
    const double a0 = 1e-6;
    double s[4] = {a0, a0, -3.0 / 7.0 * a0 * a0, -6.0 / 7.0 * a0 * a0};
    double y = std::log(a0), h = 1e-3;
    std::vector<double> raw(4 * n);
    for (size_t i = 0; i < n; ++i) {
        integrate_growth(y, std::log(tg[order[i]]), s, Om, OL, h);
        for (int q = 0; q < 4; ++q) raw[4 * order[i] + q] = s[q];
    }
    const double nm = raw[4 * (n - 1)];
    const size_t m = a.size();
    D1.resize(m);
    D2.resize(m);
    dD1da.resize(m);
    dD2da.resize(m);
    for (size_t i = 0; i < m; ++i) {
        D1[i] = raw[4 * i + 0] / nm;
        dD1da[i] = raw[4 * i + 1] / nm / a[i];
        D2[i] = raw[4 * i + 2] / (nm * nm);
        dD2da[i] = raw[4 * i + 3] / (nm * nm) / a[i];
    }
}

double alpha_tilde(double ai, double af, double aK, double Om, double OL, double nLPT) {
    auto f = [&](double a) { return std::pow(a, nLPT - 2.0) / conformal_hubble(a, Om, OL); };
    return std::pow(aK, -nLPT) * composite_gl(f, ai, af, 16, 20);
}

double beta_tilde(double ai, double af, double aD, double Om, double OL, double nLPT) {
    return -1.5 * Om * (std::pow(af, nLPT) - std::pow(ai, nLPT)) /
           (nLPT * std::pow(aD, nLPT) * conformal_hubble(aD, Om, OL));
}

// Standard factors (App. B): the drift and kick prefactors integrated over the interval.
double alpha_standard(double ai, double af, double Om, double OL) {
    auto f = [&](double a) { return 1.0 / (a * a * conformal_hubble(a, Om, OL)); };
    return composite_gl(f, ai, af, 16, 20);
}

double beta_standard(double ai, double af, double Om, double OL) {
    auto f = [&](double a) { return -1.5 * Om / (a * conformal_hubble(a, Om, OL)); };
    return composite_gl(f, ai, af, 16, 20);
}

TimeTable build_time_table(const scola_params &p) {
    TimeTable t;
    const int n = p.nsteps;
    t.a.resize(n + 1);
    for (int k = 0; k <= n; ++k) t.a[k] = p.a_i + (p.a_f - p.a_i) * k / n;
    t.a[n] = p.a_f;
    t.a_half.resize(n);
    for (int k = 0; k < n; ++k) t.a_half[k] = 0.5 * (t.a[k] + t.a[k + 1]);
    std::vector<double> q = t.a;
    q.push_back(p.a_i);
    q.push_back(p.a_f);
    std::vector<double> D1, D2, d1, d2;
    growth_factors(p.Om, p.OL, q, D1, D2, d1, d2);
    t.D1.assign(D1.begin(), D1.begin() + n + 1);
    t.D2.assign(D2.begin(), D2.begin() + n + 1);
    t.D1_i = D1[n + 1];
    t.D2_i = D2[n + 1];
    t.D1_f = D1[n + 2];
    t.D2_f = D2[n + 2];
    t.dD1da_f = d1[n + 2];
    t.dD2da_f = d2[n + 2];
    t.Hconf_f = conformal_hubble(p.a_f, p.Om, p.OL);
    t.beta.resize(n + 1);
    t.kick_from.resize(n + 1);
    t.kick_to.resize(n + 1);
    for (int k = 0; k <= n; ++k) {
        t.kick_from[k] = (k == 0) ? t.a[0] : t.a_half[k - 1];
        t.kick_to[k] = (k < n) ? t.a_half[k] : t.a[n];
        t.beta[k] = p.time_stepping == SCOLA_STEPPING_STANDARD
                        ? beta_standard(t.kick_from[k], t.kick_to[k], p.Om, p.OL)
                        : beta_tilde(t.kick_from[k], t.kick_to[k], t.a[k], p.Om, p.OL, p.nLPT);
    }
    t.alpha.resize(n);
    t.dD1.resize(n);
    t.dD2.resize(n);
    for (int k = 0; k < n; ++k) {
        t.alpha[k] = p.time_stepping == SCOLA_STEPPING_STANDARD
                         ? alpha_standard(t.a[k], t.a[k + 1], p.Om, p.OL)
                         : alpha_tilde(t.a[k], t.a[k + 1], t.a_half[k], p.Om, p.OL, p.nLPT);
        t.dD1[k] = t.D1[k + 1] - t.D1[k];
        t.dD2[k] = t.D2[k + 1] - t.D2[k];
    }
    return t;
}

double bbks_amplitude(double Om, double h, double ns, double sigma8) {
    auto f = [&](double lnk) {
        const double k = std::exp(lnk);
        const double T = bbks_T(k, Om, h);
        const double W = tophat(8.0 * k);
        return k * k * k * std::pow(k, ns) * T * T * W * W / (2.0 * M_PI * M_PI);
    };
    const double s2 = composite_gl(f, std::log(1e-5), std::log(1e3), 4000, 16);
    return sigma8 * sigma8 / s2;
}

}  // namespace scola
