// Spin-restricted exchange-correlation functionals on the device, templated on
// the arithmetic type (both forms evaluate them in double: float32 PBE was measured
// too inaccurate for the mixed form's bound).  Each returns the energy per volume f = rho*eps and the first
// derivatives vrho = df/drho and vsigma = df/dsigma with sigma = |grad rho|^2,
// the reading of Eqs. zvec_r / z_mat under which V_xc = dE_xc/dP.
//
// Slater exchange: f = C_x rho^(4/3), C_x = -(3/4)(3/pi)^(1/3).
// PBE exchange:    f = C_x rho^(4/3) F_x(s^2), F_x = 1 + kappa - kappa/(1 + mu s^2/kappa),
//                  s^2 = sigma / (4 (3 pi^2)^(2/3) rho^(8/3)).
// PBE correlation: f = rho (eps_PW92(r_s) + H), r_s = (3/(4 pi rho))^(1/3),
//                  t^2 = pi sigma / (16 (3 pi^2)^(1/3) rho^(7/3)),
//                  H = gamma ln(1 + (beta/gamma) t^2 (1 + A t^2)/(1 + A t^2 + A^2 t^4)),
//                  A = (beta/gamma)/(exp(-eps/gamma) - 1).
// PW92 (unpolarised): eps = -2a(1 + a1 r_s) ln(1 + 1/(2a Q)),
//                  Q = b1 r_s^(1/2) + b2 r_s + b3 r_s^(3/2) + b4 r_s^2.
// PBE0, semi-local part: f = (1 - a) f_x^PBE + f_c^PBE with a = 1/4, the exact-exchange
//                  fraction of the hybrid; the a E_x^HF term is a four-centre integral over the
//                  orbitals, not a grid quadrature, and belongs to the caller's exchange code.
// Derivatives are written out by the chain rule, term by term.
#pragma once

namespace gbxc {
namespace xc {

constexpr double kRhoMin = 1e-15;
constexpr double kCx = -0.7385587663820223;          // -(3/4)(3/pi)^(1/3)
constexpr double kS2Scale = 0.026121172985233605;     // 1 / (4 (3 pi^2)^(2/3))
constexpr double kRsScale = 0.6203504908994001;       // (3/(4 pi))^(1/3)
constexpr double kT2Scale = 0.0634682060977037;       // pi / (16 (3 pi^2)^(1/3))
constexpr double kKappa = 0.804;
constexpr double kBeta = 0.06672455060314922;
constexpr double kMu = 0.21951497276451704;           // beta pi^2 / 3
constexpr double kGamma = 0.0310906908696549;         // (1 - ln 2)/pi^2
constexpr double kPbe0ExactFraction = 0.25;           // a of PBE0
constexpr double kPwA = 0.031091, kPwA1 = 0.21370;
constexpr double kPwB1 = 7.5957, kPwB2 = 3.5876, kPwB3 = 1.6382, kPwB4 = 0.49294;

__device__ __forceinline__ double m_cbrt(double v) { return cbrt(v); }
__device__ __forceinline__ float m_cbrt(float v) { return cbrtf(v); }
__device__ __forceinline__ double m_sqrt(double v) { return sqrt(v); }
__device__ __forceinline__ float m_sqrt(float v) { return sqrtf(v); }
__device__ __forceinline__ double m_exp(double v) { return exp(v); }
__device__ __forceinline__ float m_exp(float v) { return expf(v); }
__device__ __forceinline__ double m_expm1(double v) { return expm1(v); }
__device__ __forceinline__ float m_expm1(float v) { return expm1f(v); }
__device__ __forceinline__ double m_log1p(double v) { return log1p(v); }
__device__ __forceinline__ float m_log1p(float v) { return log1pf(v); }

template <typename T>
__device__ __forceinline__ void slater(T rho, T &f, T &vrho, T &vsigma) {
    T r13 = m_cbrt(rho);
    f = T(kCx) * rho * r13;
    vrho = T(4.0 / 3.0) * T(kCx) * r13;
    vsigma = T(0);
}

template <typename T>
__device__ __forceinline__ void pbe_x(T rho, T sigma, T &f, T &vrho, T &vsigma) {
    T r13 = m_cbrt(rho);
    T r43 = rho * r13;
    T ds2 = T(kS2Scale) / (r43 * r43);      // d s^2 / d sigma
    T s2 = sigma * ds2;
    T den = T(1) + T(kMu / kKappa) * s2;
    T Fx = T(1) + T(kKappa) - T(kKappa) / den;
    T dFx = T(kMu) / (den * den);           // dF_x / d s^2
    f = T(kCx) * r43 * Fx;
    vrho = T(4.0 / 3.0) * T(kCx) * r13 * Fx - T(8.0 / 3.0) * T(kCx) * r13 * dFx * s2;
    vsigma = T(kCx) * r43 * dFx * ds2;
}

template <typename T>
__device__ __forceinline__ void pbe_c(T rho, T sigma, T &f, T &vrho, T &vsigma) {
    T r13 = m_cbrt(rho);
    T rs = T(kRsScale) / r13;
    T srs = m_sqrt(rs);
    T Q = T(kPwB1) * srs + T(kPwB2) * rs + T(kPwB3) * rs * srs + T(kPwB4) * rs * rs;
    T dQ = T(0.5 * kPwB1) / srs + T(kPwB2) + T(1.5 * kPwB3) * srs + T(2.0 * kPwB4) * rs;
    T lg = m_log1p(T(1) / (T(2.0 * kPwA) * Q));
    T eps = T(-2.0 * kPwA) * (T(1) + T(kPwA1) * rs) * lg;
    T deps_drs = T(-2.0 * kPwA * kPwA1) * lg +
                 T(2.0 * kPwA) * (T(1) + T(kPwA1) * rs) * dQ / (Q * (T(2.0 * kPwA) * Q + T(1)));
    T deps_drho = deps_drs * (-rs / (T(3) * rho));
    T Em1 = m_expm1(-eps / T(kGamma));      // exp(-eps/gamma) - 1 without cancellation
    T E = Em1 + T(1);
    T A = T(kBeta / kGamma) / Em1;
    T dA_deps = A * A * E / T(kBeta);
    T du_dsigma = T(kT2Scale) / (rho * rho * r13);
    T u = sigma * du_dsigma;                 // t^2
    T Au = A * u;
    T num = u + Au * u;
    T den = T(1) + Au + Au * Au;
    T inv_den2 = T(1) / (den * den);
    T Y = num / den;
    T dY_du = ((T(1) + T(2) * Au) * den - num * (A + T(2) * A * Au)) * inv_den2;
    T dY_dA = (u * u * den - num * (u + T(2) * Au * u)) * inv_den2;
    T H = T(kGamma) * m_log1p(T(kBeta / kGamma) * Y);
    T dH_dY = T(kBeta) / (T(1) + T(kBeta / kGamma) * Y);
    T du_drho = T(-7.0 / 3.0) * u / rho;
    T dH_drho = dH_dY * (dY_du * du_drho + dY_dA * dA_deps * deps_drho);
    f = rho * (eps + H);
    vrho = eps + H + rho * (deps_drho + dH_drho);
    vsigma = rho * dH_dY * dY_du * du_dsigma;
}

// Evaluate functional `fn` (GBXC_SLATER, GBXC_PBE or GBXC_PBE0_SL); zero below kRhoMin.
template <typename T>
__device__ __forceinline__ void evaluate(int fn, T rho, T sigma, T &f, T &vrho, T &vsigma) {
    if (!(rho >= T(kRhoMin))) {
        f = vrho = vsigma = T(0);
        return;
    }
    if (fn == GBXC_SLATER) {
        slater(rho, f, vrho, vsigma);
    } else {
        T fx, vx, sx, fc, vc, sc;
        pbe_x(rho, sigma, fx, vx, sx);
        pbe_c(rho, sigma, fc, vc, sc);
        if (fn == GBXC_PBE0_SL) {   // the hybrid's semi-local part: (1 - a) PBE exchange
            const T k = T(1) - T(kPbe0ExactFraction);
            fx *= k;
            vx *= k;
            sx *= k;
        }
        f = fx + fc;
        vrho = vx + vc;
        vsigma = sx + sc;
    }
}

// ---------------------------------------------------------------- spin-polarised forms
// Arguments rho_a, rho_b, sigma_aa, sigma_ab, sigma_bb; results f and its derivatives
// va, vb (rho_a, rho_b), saa, sab, sbb (the three sigmas).
//
// Exchange by spin scaling, f = f(2 rho_a, 4 sigma_aa)/2 + f(2 rho_b, 4 sigma_bb)/2.
// PBE correlation with the PW92 spin interpolation (Perdew and Wang 1992):
//   eps_c = e0 + alpha_c f(zeta)(1 - zeta^4)/f''(0) + (e1 - e0) f(zeta) zeta^4,
//   f(zeta) = ((1+zeta)^(4/3) + (1-zeta)^(4/3) - 2)/(2^(4/3) - 2),
//   e0, e1, -alpha_c = G(r_s) with PW92's three parameter sets,
//   H = gamma phi^3 ln(1 + (beta/gamma) Y(t^2, A)), phi = ((1+zeta)^(2/3) + (1-zeta)^(2/3))/2,
//   t^2 = pi sigma/(16 (3 pi^2)^(1/3) rho^(7/3) phi^2), A = (beta/gamma)/(exp(-eps_c/(gamma phi^3)) - 1),
// with rho = rho_a + rho_b, zeta = (rho_a - rho_b)/rho clamped to |zeta| <= 1 - 1e-10 and
// sigma = sigma_aa + 2 sigma_ab + sigma_bb; zero below rho = kRhoMin.
constexpr double kZetaMax = 1.0 - 1e-10;
constexpr double kFzDen = 0.5198420997897464;          // 2^(4/3) - 2
constexpr double kFpp0 = 1.7099209341613653;           // 8 / (9 (2^(4/3) - 2))
// PW92's parameter sets: 0 = e0 (paramagnetic), 1 = e1 (ferromagnetic), 2 = -alpha_c
template <int K>
struct PwSet;
template <>
struct PwSet<0> {
    static constexpr double A = 0.031091, a1 = 0.21370, b1 = 7.5957, b2 = 3.5876, b3 = 1.6382, b4 = 0.49294;
};
template <>
struct PwSet<1> {
    static constexpr double A = 0.015545, a1 = 0.20548, b1 = 14.1189, b2 = 6.1977, b3 = 3.3662, b4 = 0.62517;
};
template <>
struct PwSet<2> {
    static constexpr double A = 0.016887, a1 = 0.11125, b1 = 10.357, b2 = 3.6231, b3 = 0.88026, b4 = 0.49671;
};

template <int K, typename T>
__device__ __forceinline__ void pw_G(T rs, T &g, T &dg) {
    using p = PwSet<K>;
    T srs = m_sqrt(rs);
    T Q = T(p::b1) * srs + T(p::b2) * rs + T(p::b3) * rs * srs + T(p::b4) * rs * rs;
    T dQ = T(0.5 * p::b1) / srs + T(p::b2) + T(1.5 * p::b3) * srs + T(2.0 * p::b4) * rs;
    T lg = m_log1p(T(1) / (T(2.0 * p::A) * Q));
    g = T(-2.0 * p::A) * (T(1) + T(p::a1) * rs) * lg;
    dg = T(-2.0 * p::A * p::a1) * lg + T(2.0 * p::A) * (T(1) + T(p::a1) * rs) * dQ / (Q * (T(2.0 * p::A) * Q + T(1)));
}

template <typename T>
__device__ __forceinline__ void pbe_c_pol(T ra, T rb, T saa, T sab, T sbb, T &f, T &va, T &vb, T &s_aa, T &s_ab,
                                          T &s_bb) {
    const T rho = ra + rb;
    if (!(rho >= T(kRhoMin))) {
        f = va = vb = s_aa = s_ab = s_bb = T(0);
        return;
    }
    T zeta = (ra - rb) / rho;
    zeta = zeta > T(kZetaMax) ? T(kZetaMax) : (zeta < T(-kZetaMax) ? T(-kZetaMax) : zeta);
    const T sig = saa + T(2) * sab + sbb;
    const T r13 = m_cbrt(rho);
    const T rs = T(kRsScale) / r13;
    T e0, de0, e1, de1, mac, dmac;
    pw_G<0>(rs, e0, de0);
    pw_G<1>(rs, e1, de1);
    pw_G<2>(rs, mac, dmac);
    const T opz = T(1) + zeta, omz = T(1) - zeta;
    const T co = m_cbrt(opz), cm = m_cbrt(omz);
    const T fz = (opz * co + omz * cm - T(2)) / T(kFzDen);
    const T dfz = T(4.0 / 3.0) * (co - cm) / T(kFzDen);
    const T z2 = zeta * zeta, z3 = z2 * zeta, z4 = z2 * z2;
    const T eps = e0 - mac * fz * (T(1) - z4) / T(kFpp0) + (e1 - e0) * fz * z4;
    const T deps_drs = de0 - dmac * fz * (T(1) - z4) / T(kFpp0) + (de1 - de0) * fz * z4;
    const T deps_dz = -mac * (dfz * (T(1) - z4) - T(4) * z3 * fz) / T(kFpp0) + (e1 - e0) * (dfz * z4 + T(4) * z3 * fz);
    const T deps_drho = deps_drs * (-rs / (T(3) * rho));
    const T phi = T(0.5) * (co * co + cm * cm);
    const T dphi = T(1.0 / 3.0) * (T(1) / co - T(1) / cm);
    const T phi2 = phi * phi, phi3 = phi2 * phi;
    const T Em1 = m_expm1(-eps / (T(kGamma) * phi3));
    const T E = Em1 + T(1);
    const T A = T(kBeta / kGamma) / Em1;
    const T dA_deps = A * A * E / (T(kBeta) * phi3);
    const T dA_dphi = T(-3) * A * A * E * eps / (T(kBeta) * phi3 * phi);
    const T du_dsig = T(kT2Scale) / (rho * rho * r13 * phi2);
    const T u = sig * du_dsig;   // t^2
    const T Au = A * u;
    const T num = u + Au * u;
    const T den = T(1) + Au + Au * Au;
    const T inv_den2 = T(1) / (den * den);
    const T Y = num / den;
    const T dY_du = ((T(1) + T(2) * Au) * den - num * (A + T(2) * A * Au)) * inv_den2;
    const T dY_dA = (u * u * den - num * (u + T(2) * Au * u)) * inv_den2;
    const T Lg = m_log1p(T(kBeta / kGamma) * Y);
    const T dL_dY = T(kBeta / kGamma) / (T(1) + T(kBeta / kGamma) * Y);
    const T gp3 = T(kGamma) * phi3;
    const T H = gp3 * Lg;
    const T du_drho = T(-7.0 / 3.0) * u / rho;
    const T du_dphi = T(-2) * u / phi;
    const T dH_drho = gp3 * dL_dY * (dY_du * du_drho + dY_dA * dA_deps * deps_drho);
    const T dH_dz = T(3) * T(kGamma) * phi2 * dphi * Lg +
                    gp3 * dL_dY * (dY_du * du_dphi * dphi + dY_dA * (dA_deps * deps_dz + dA_dphi * dphi));
    const T dH_dsig = gp3 * dL_dY * dY_du * du_dsig;
    f = rho * (eps + H);
    const T df_drho = eps + H + rho * (deps_drho + dH_drho);
    const T df_dz = rho * (deps_dz + dH_dz);
    va = df_drho + (T(1) - zeta) / rho * df_dz;
    vb = df_drho - (T(1) + zeta) / rho * df_dz;
    s_aa = s_bb = rho * dH_dsig;
    s_ab = T(2) * rho * dH_dsig;
}

// one spin channel of a spin-scaled exchange
template <typename T>
__device__ __forceinline__ void exchange_channel(int fn, T r, T s, T &f, T &v, T &vs) {
    T ff = T(0), vr = T(0), vsg = T(0);
    if (T(2) * r >= T(kRhoMin)) {
        if (fn == GBXC_SLATER) slater(T(2) * r, ff, vr, vsg);
        else pbe_x(T(2) * r, T(4) * s, ff, vr, vsg);
    }
    const T k = fn == GBXC_PBE0_SL ? T(1) - T(kPbe0ExactFraction) : T(1);
    f = T(0.5) * k * ff;
    v = k * vr;
    vs = T(2) * k * vsg;
}

template <typename T>
__device__ __forceinline__ void evaluate_pol(int fn, T ra, T rb, T saa, T sab, T sbb, T &f, T &va, T &vb, T &s_aa,
                                             T &s_ab, T &s_bb) {
    T fa, fb, xa, xb, xsa, xsb;
    exchange_channel(fn, ra, saa, fa, xa, xsa);
    exchange_channel(fn, rb, sbb, fb, xb, xsb);
    f = fa + fb;
    va = xa;
    vb = xb;
    s_aa = xsa;
    s_ab = T(0);
    s_bb = xsb;
    if (fn == GBXC_PBE || fn == GBXC_PBE0_SL) {
        T fc, ca, cb, csa, csab, csb;
        pbe_c_pol(ra, rb, saa, sab, sbb, fc, ca, cb, csa, csab, csb);
        f += fc;
        va += ca;
        vb += cb;
        s_aa += csa;
        s_ab += csab;
        s_bb += csb;
    }
}

// ---- meta-GGA: MVS exchange (Sun, Perdew and Ruzsinszky 2015), spin-restricted, float64.
//   f = C_x rho^(4/3) (1 + kappa0 f_a(alpha)) / (1 + b s^4)^(1/8),
//   f_a = (1 - alpha) / ((1 + e1 alpha^2)^2 + c1 alpha^4)^(1/4),
//   alpha = (tau - sigma/(8 rho)) / tau_unif, tau_unif = (3/10)(3 pi^2)^(2/3) rho^(5/3),
//   kappa0 = 0.174, e1 = -1.6665, c1 = 0.7438, b = 0.0233;
// returns f and its derivatives with respect to rho, sigma and tau (zero below kRhoMin).
constexpr double kMvsKappa0 = 0.174, kMvsE1 = -1.6665, kMvsC1 = 0.7438, kMvsB = 0.0233;
constexpr double kTauUnif = 2.871234000188191;        // (3/10)(3 pi^2)^(2/3)

__device__ __forceinline__ void mvs_x(double rho, double sigma, double tau, double &f, double &vrho, double &vsigma,
                                      double &vtau) {
    f = vrho = vsigma = vtau = 0.0;
    if (!(rho >= kRhoMin)) return;
    const double r13 = cbrt(rho), r53 = rho * r13 * r13;
    const double u = kS2Scale * sigma / (r53 * rho);                 // s^2
    const double at = 1.0 / (kTauUnif * r53);                        // d alpha / d tau
    const double al = (tau - sigma / (8.0 * rho)) * at;
    const double q = 1.0 + kMvsE1 * al * al;
    const double D = q * q + kMvsC1 * al * al * al * al;
    const double D14 = sqrt(sqrt(D));                                 // D^(1/4)
    const double fa = (1.0 - al) / D14;
    const double dD = 4.0 * kMvsE1 * al * q + 4.0 * kMvsC1 * al * al * al;
    const double dfa = -1.0 / D14 - 0.25 * (1.0 - al) * dD / (D * D14);
    const double p = 1.0 + kMvsB * u * u;
    const double g = 1.0 / sqrt(sqrt(sqrt(p)));                       // p^(-1/8)
    const double dg = -0.25 * kMvsB * u * g / p;
    const double F = (1.0 + kMvsKappa0 * fa) * g;
    const double Fu = (1.0 + kMvsKappa0 * fa) * dg;
    const double Fa = kMvsKappa0 * dfa * g;
    const double ur = -(8.0 / 3.0) * u / rho, us = kS2Scale / (r53 * rho);
    const double as = -at / (8.0 * rho), ar = sigma / (8.0 * rho * rho) * at - (5.0 / 3.0) * al / rho;
    const double e0 = kCx * rho * r13;
    f = e0 * F;
    vrho = (4.0 / 3.0) * kCx * r13 * F + e0 * (Fu * ur + Fa * ar);
    vsigma = e0 * (Fu * us + Fa * as);
    vtau = e0 * Fa * at;
}

}  // namespace xc
}  // namespace gbxc
