// Spin-restricted exchange-correlation functionals on the device, templated on
// the arithmetic type (double for the float64 form, float for the bulk of the
// mixed form).  Each returns the energy per volume f = rho*eps and the first
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

// Evaluate functional `fn` (GBXC_SLATER or GBXC_PBE); zero below kRhoMin.
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
        f = fx + fc;
        vrho = vx + vc;
        vsigma = sx + sc;
    }
}

}  // namespace xc
}  // namespace gbxc
