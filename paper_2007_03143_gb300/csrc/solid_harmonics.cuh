// Pure (spherical) shells: the 2L+1 real solid harmonics S_Lm, m = -L..L, in Racah
// normalisation (sqrt(4 pi/(2L+1)) r^L Y_Lm, the same norm on the sphere as x^L) as
// combinations of a shell's Cartesian functions, for L = 2 and 3 (the paper's cc-pVDZ runs
// use spherical d functions, Sec. 3).  Input order is the Cartesian component order
// (l descending, then m descending); output order m = -L..L.
//
//   L = 2:  sqrt3 xy, sqrt3 yz, z^2 - (x^2 + y^2)/2, sqrt3 xz, sqrt3/2 (x^2 - y^2)
//   L = 3:  A (3 x^2 y - y^3), sqrt15 xyz, B (4 y z^2 - x^2 y - y^3), z^3 - 3/2 (x^2 z + y^2 z),
//           B (4 x z^2 - x^3 - x y^2), sqrt15/2 (x^2 z - y^2 z), A (x^3 - 3 x y^2)
//           with A = sqrt(5/8), B = sqrt(3/8)
//
// The arithmetic is a policy (Ops::add, Ops::sub, Ops::scale by a double constant) so the
// float64 and the double-float collocation share the combinations.
#pragma once

namespace gbxc {
namespace sph {

constexpr double kS3 = 1.7320508075688772935;    // sqrt(3)
constexpr double kS15 = 3.8729833462074168852;   // sqrt(15)
constexpr double kA = 0.79056941504209483300;    // sqrt(5/8)
constexpr double kB = 0.61237243569579452455;    // sqrt(3/8)

template <class Ops, typename T>
__device__ __forceinline__ void pure2(const T *c, T *o) {
    // c: xx xy xz yy yz zz
    o[0] = Ops::scale(c[1], kS3);
    o[1] = Ops::scale(c[4], kS3);
    o[2] = Ops::sub(c[5], Ops::scale(Ops::add(c[0], c[3]), 0.5));
    o[3] = Ops::scale(c[2], kS3);
    o[4] = Ops::scale(Ops::sub(c[0], c[3]), 0.5 * kS3);
}

template <class Ops, typename T>
__device__ __forceinline__ void pure3(const T *c, T *o) {
    // c: xxx xxy xxz xyy xyz xzz yyy yyz yzz zzz
    o[0] = Ops::scale(Ops::sub(Ops::scale(c[1], 3.0), c[6]), kA);
    o[1] = Ops::scale(c[4], kS15);
    o[2] = Ops::scale(Ops::sub(Ops::scale(c[8], 4.0), Ops::add(c[1], c[6])), kB);
    o[3] = Ops::sub(c[9], Ops::scale(Ops::add(c[2], c[7]), 1.5));
    o[4] = Ops::scale(Ops::sub(Ops::scale(c[5], 4.0), Ops::add(c[0], c[3])), kB);
    o[5] = Ops::scale(Ops::sub(c[2], c[7]), 0.5 * kS15);
    o[6] = Ops::scale(Ops::sub(c[0], Ops::scale(c[3], 3.0)), kA);
}

// out (2L+1 values) from the (L+1)(L+2)/2 Cartesian values, L = 2 or 3
template <int L, class Ops, typename T>
__device__ __forceinline__ void pure(const T *c, T *o) {
    static_assert(L == 2 || L == 3, "pure shells are built for L = 2 and 3");
    if constexpr (L == 2) pure2<Ops>(c, o);
    else pure3<Ops>(c, o);
}

struct DoubleOps {
    __device__ static double add(double a, double b) { return a + b; }
    __device__ static double sub(double a, double b) { return a - b; }
    __device__ static double scale(double a, double k) { return a * k; }
};

}  // namespace sph
}  // namespace gbxc
