// Host-side pole expansion of the Fermi-Dirac function (md_make_poles).
//
// g(eps) = 1/(1+exp((eps-mu)/kT)) (the paper's Eq. (dm)) is approximated on
// [emin, emax] by r(eps) = sum_p Im(w_p/(eps - z_p)), Im z_p > 0.
//
// Construction (Hale, Higham & Trefethen, SIAM J. Numer. Anal. 46 (2008)
// contour quadrature; square-root substitution of Lin, Lu, Ying & E,
// Chin. Ann. Math. 30B (2009)).  With x = eps - mu, a = (pi kT)^2 and the
// spectrum in x in [-dE, dE]:
//   * write g(x) as a Cauchy integral over a closed curve around [-dE, dE]
//     threading between the Matsubara poles +-i pi kT;
//   * substitute w = xi^2 + a: the curve becomes one closed curve around
//     [m, M] = [a, dE^2 + a] and the integrand the even function
//     F(w) = (g(xi)/(xi - x) + g(-xi)/(xi + x)) / (2 xi);
//   * map the strip 0 < Im t < K' conformally onto C \ ((-inf,0] U [m,M])
//     by w(t) = sqrt(mM) (1/k + sn t)/(1/k - sn t),
//     k = (sqrt M - sqrt m)/(sqrt M + sqrt m);
//   * trapezoid rule with N = P nodes on Im t = K'/2, period 4K; conjugate
//     symmetry leaves N/2 nodes, each giving two poles:
//         z = mu + xi_j,        w = c_j g(xi_j)
//         z = mu - conj(xi_j),  w = conj(c_j g(-xi_j)),
//     c_j = h w'(t_j) / (2 pi xi_j), h = 4K/N.
// The entropy term of Eq. (tot) uses the same nodes with the weights of its
// own function phi_S (md_make_entropy_weights): the construction needs no
// more of g than its analyticity off the Matsubara rays, and phi_S has its
// singularities at the same points.
// Elliptic functions: K from the arithmetic-geometric mean (A&S 17.6),
// sn/cn/dn of a real argument from the AGM / descending Landen scheme
// (A&S 16.4), of a complex argument from the addition formulas
// (A&S 16.21.1-3).
#include <cmath>
#include <complex>
#include <string>

#include "md_internal.h"

namespace md {

namespace {

using cd = std::complex<double>;
constexpr double kPi = 3.14159265358979323846;

double agm(double a, double b) {
    for (int it = 0; it < 64; ++it) {
        const double an = 0.5 * (a + b);
        const double bn = std::sqrt(a * b);
        a = an;
        b = bn;
        if (std::fabs(a - b) <= 1e-16 * a) break;
    }
    return 0.5 * (a + b);
}

// K(k) given k' = sqrt(1 - k^2): K = pi / (2 AGM(1, k')).
double complete_K_from_kprime(double kprime) { return kPi / (2.0 * agm(1.0, kprime)); }

// sn, cn, dn of real u for parameter m = k^2 (0 <= m < 1), A&S 16.4.
void jacobi_real(double u, double m, double& sn, double& cn, double& dn) {
    if (m == 0.0) {
        sn = std::sin(u);
        cn = std::cos(u);
        dn = 1.0;
        return;
    }
    double a[40], c[40];
    a[0] = 1.0;
    double b = std::sqrt(1.0 - m);
    c[0] = std::sqrt(m);
    int n = 0;
    while (n < 38 && std::fabs(c[n]) > 1e-17) {
        const double an = 0.5 * (a[n] + b);
        const double cn1 = 0.5 * (a[n] - b);
        b = std::sqrt(a[n] * b);
        ++n;
        a[n] = an;
        c[n] = cn1;
    }
    double phi = std::ldexp(a[n] * u, n);
    double phi_prev = phi;
    for (int i = n; i >= 1; --i) {
        phi_prev = phi;
        phi = 0.5 * (phi + std::asin(c[i] * std::sin(phi) / a[i]));
    }
    sn = std::sin(phi);
    cn = std::cos(phi);
    dn = (n >= 1) ? cn / std::cos(phi_prev - phi) : 1.0;
}

// sn, cn, dn of complex t = x + i y, parameter m (m1 = 1 - m), A&S 16.21.
void jacobi_complex(cd t, double m, double m1, cd& sn, cd& cn, cd& dn) {
    double s, c, d, s1, c1, d1;
    jacobi_real(t.real(), m, s, c, d);
    jacobi_real(t.imag(), m1, s1, c1, d1);
    const double den = c1 * c1 + m * s * s * s1 * s1;
    sn = cd(s * d1, c * d * s1 * c1) / den;
    cn = cd(c * c1, -s * d * s1 * d1) / den;
    dn = cd(d * c1 * d1, -m * s * c * s1) / den;
}

// Fermi-Dirac function at complex x (kT > 0), free of overflow.
cd fermi_c(cd x, double kT) {
    if (x.real() > 0.0) {
        const cd e = std::exp(-x / kT);
        return e / (1.0 + e);
    }
    return 1.0 / (1.0 + std::exp(x / kT));
}

// ln(1 + u) for complex |u| < 1 that stays accurate for tiny |u| (forming
// 1 + u first would lose the digits of u): the alternating Taylor series to
// order 16 where |u| < 0.1 (remainder below 0.1^17 / 17), the logarithm of
// 1 + u elsewhere.
cd log1p_c(cd u) {
    if (std::abs(u) < 0.1) {
        cd acc = 0.0;
        for (int k = 16; k >= 1; --k) acc = u * ((k % 2 ? 1.0 : -1.0) / k + acc);
        return acc;
    }
    return std::log(1.0 + u);
}

// Entropy function of the last term of Eq. (tot), phi_S(x) = -[f ln f +
// (1-f) ln(1-f)] with f the Fermi-Dirac function, continued analytically off
// the imaginary rays where its branch points (the Matsubara points) lie.
// With y = x/kT: phi_S = ln(1 + e^y) - (1 - f) y, evaluated in the
// half-plane form that keeps the exponential below one in modulus:
//   Re y > 0:  ln(1 + e^-y) + y e^-y / (1 + e^-y)
//   else:      ln(1 + e^y)  - y e^y  / (1 + e^y)
cd entropy_c(cd x, double kT) {
    const cd y = x / kT;
    if (y.real() > 0.0) {
        const cd e = std::exp(-y);
        return log1p_c(e) + y * e / (1.0 + e);
    }
    const cd e = std::exp(y);
    return log1p_c(e) - y * e / (1.0 + e);
}

// Trapezoid nodes of the construction above, with the weights of the
// function phi(x, kT): node j gives the poles mu + xi_j (weight c_j phi(xi_j))
// and mu - conj(xi_j) (weight conj(c_j phi(-xi_j))).
md_status contour_poles(cd (*phi)(cd, double), const char* who, double kT, double mu, double emin,
                        double emax, int P, double* z_out, double* w_out) {
    if (!(kT > 0.0) || !(emax > emin) || !std::isfinite(mu) || !std::isfinite(emin) ||
        !std::isfinite(emax))
        return set_error(MD_ERR_INVALID, std::string(who) + ": need kT > 0, finite mu and emin < emax");
    if (P < 2 || (P % 2) != 0) return set_error(MD_ERR_INVALID, std::string(who) + ": P must be even and >= 2");
    if (!w_out) return set_error(MD_ERR_INVALID, std::string(who) + ": null output");
    const double dE = std::fmax(std::fabs(emin - mu), std::fabs(emax - mu));
    const double a = (kPi * kT) * (kPi * kT);
    const double lo = a, hi = dE * dE + a;
    const double sl = std::sqrt(lo), sh = std::sqrt(hi);
    const double k = (sh - sl) / (sh + sl);
    const double one_minus_k = 2.0 * sl / (sh + sl);
    const double kp2 = one_minus_k * (1.0 + k);  // 1 - k^2 without cancellation
    const double kp = std::sqrt(kp2);
    const double K = complete_K_from_kprime(kp);   // K(k)
    const double Kp = complete_K_from_kprime(k);   // K(k') : its complementary modulus is k
    const double h = 4.0 * K / P;
    const double c0 = std::sqrt(lo * hi);
    for (int j = 0; j < P / 2; ++j) {
        const cd t(-K + (j + 0.5) * h, 0.5 * Kp);
        cd sn, cn, dn;
        jacobi_complex(t, k * k, kp2, sn, cn, dn);
        const cd den = 1.0 / k - sn;
        const cd wq = c0 * (1.0 / k + sn) / den;
        const cd dw = c0 * (2.0 / k) * cn * dn / (den * den);
        const cd xi = std::sqrt(wq - a);
        const cd cj = h * dw / (2.0 * kPi * xi);
        const cd wa = cj * phi(xi, kT);
        const cd wb = std::conj(cj * phi(-xi, kT));
        if (z_out) {
            const cd za = mu + xi;
            const cd zb = mu - std::conj(xi);
            z_out[4 * j + 0] = za.real();
            z_out[4 * j + 1] = za.imag();
            z_out[4 * j + 2] = zb.real();
            z_out[4 * j + 3] = zb.imag();
        }
        w_out[4 * j + 0] = wa.real();
        w_out[4 * j + 1] = wa.imag();
        w_out[4 * j + 2] = wb.real();
        w_out[4 * j + 3] = wb.imag();
    }
    return MD_OK;
}

}  // namespace

md_status make_entropy_weights(double kT, double mu, double emin, double emax, int P, double* w_out) {
    return contour_poles(entropy_c, "md_make_entropy_weights", kT, mu, emin, emax, P, nullptr, w_out);
}

md_status make_poles(double kT, double mu, double emin, double emax, int P, double* z_out,
                     double* w_out) {
    if (!z_out) return set_error(MD_ERR_INVALID, "md_make_poles: null output");
    return contour_poles(fermi_c, "md_make_poles", kT, mu, emin, emax, P, z_out, w_out);
}

}  // namespace md
