// FP64 Bessel functions J0, Y0, J1, Y1 (the Hankel functions H_nu^(1) = J_nu + i Y_nu
// of G(x, y) = (i/4) H0^(1)(omega |x - y|), paper Section 1), written from two
// published methods and tested against scipy / mpmath values:
//
//  x >= 20: Hankel's asymptotic expansion (Abramowitz & Stegun 9.2.5, 9.2.9,
//           9.2.10):  H_nu^(1)(x) = sqrt(2/(pi x)) (P + i Q) exp(i chi),
//           chi = x - (nu/2 + 1/4) pi,  P = sum_k (-1)^k a_2k x^-2k,
//           Q = sum_k (-1)^k a_(2k+1) x^-(2k+1),
//           a_k(nu) = prod_{m=1..k} (4 nu^2 - (2m-1)^2) / (8^k k!).
//           Twenty-one terms reach double precision for x >= 20.
//  x <  20: Miller's backward recurrence J_(k-1) = (2k/x) J_k - J_(k+1) from
//           k = N ~ x + 36, normalised by J_0 + 2 sum_k J_2k = 1 (A&S 9.1.46),
//           then Neumann's series (A&S 9.1.88)
//             Y0 = (2/pi) [(ln(x/2) + gamma) J0 - 2 sum_k (-1)^k J_2k / k]
//           and its derivative (Y1 = -Y0')
//             Y1 = (2/pi) [(ln(x/2) + gamma) J1 - J0 / x
//                          + sum_k (-1)^k (J_(2k-1) - J_(2k+1)) / k].
#pragma once

namespace h64 {

// a_k(nu) of the asymptotic expansion with the alternating sign folded in
static __constant__ double kP0[11] = {1.0, -0.0703125, 0.112152099609375, -0.5725014209747314,
                               6.074042001273483, -110.01714026924674, 3038.090510922384,
                               -118838.42625678325, 6252951.493434797, -425939216.5047669,
                               36468400807.06556};
static __constant__ double kQ0[10] = {-0.125, 0.0732421875, -0.22710800170898438, 1.7277275025844574,
                               -24.380529699556064, 551.3358961220206, -18257.755474293175,
                               832859.3040162893, -50069589.531988926, 3836255180.2304335};
static __constant__ double kP1[11] = {1.0, 0.1171875, -0.144195556640625, 0.6765925884246826,
                               -6.883914268109947, 121.59789187653587, -3302.2722944808525,
                               127641.2726461746, -6656367.718817688, 450278600.3050393,
                               -38338575207.427895};
static __constant__ double kQ1[10] = {0.375, -0.1025390625, 0.2775764465332031, -1.993531733751297,
                               27.248827311268542, -603.8440767050702, 19718.37591223663,
                               -890297.8767070678, 53104110.10968523, -4043620325.107754};

// 2 pi = C1 + C2 + C3 with C1 on 30 significant bits (k * C1 exact for k < 2^23)
constexpr double kC1 = 6.283185310661793;
constexpr double kC2 = -3.4822062782016664e-09;
constexpr double kC3 = 6.578502774529703e-26;
constexpr double kPi4 = 0.7853981633974483;
constexpr double kPi4Lo = 3.061616997868383e-17;
constexpr double kInv2Pi = 0.15915494309189535;
constexpr double kTwoOverPi = 0.6366197723675814;
constexpr double kGamma = 0.57721566490153286061;

// 1/m for the Neumann sums (m <= 28 for x < 20)
static __constant__ double kInvM[32] = {0.0,      1.0,      1.0 / 2,  1.0 / 3,  1.0 / 4,  1.0 / 5,
                                 1.0 / 6,  1.0 / 7,  1.0 / 8,  1.0 / 9,  1.0 / 10, 1.0 / 11,
                                 1.0 / 12, 1.0 / 13, 1.0 / 14, 1.0 / 15, 1.0 / 16, 1.0 / 17,
                                 1.0 / 18, 1.0 / 19, 1.0 / 20, 1.0 / 21, 1.0 / 22, 1.0 / 23,
                                 1.0 / 24, 1.0 / 25, 1.0 / 26, 1.0 / 27, 1.0 / 28, 1.0 / 29,
                                 1.0 / 30, 1.0 / 31};

__device__ __forceinline__ void asymptotic(double x, double& J0, double& Y0, double& J1,
                                           double& Y1) {
  const double t = 1.0 / x;
  const double t2 = t * t;
  double P0 = kP0[10], P1 = kP1[10], Q0 = kQ0[9], Q1 = kQ1[9];
#pragma unroll
  for (int k = 9; k >= 0; --k) {
    P0 = fma(P0, t2, kP0[k]);
    P1 = fma(P1, t2, kP1[k]);
  }
#pragma unroll
  for (int k = 8; k >= 0; --k) {
    Q0 = fma(Q0, t2, kQ0[k]);
    Q1 = fma(Q1, t2, kQ1[k]);
  }
  Q0 *= t;
  Q1 *= t;
  const double amp = sqrt(kTwoOverPi * t);
  // chi = x - pi/4 reduced to [-pi, pi] (Cody-Waite, three-part 2 pi)
  const double k = rint(fma(x, kInv2Pi, -0.125));
  double chi = fma(-k, kC1, x);
  chi = fma(-k, kC2, chi);
  chi = (chi - kPi4) - kPi4Lo;
  chi = fma(-k, kC3, chi);
  double s, c;
  sincos(chi, &s, &c);
  J0 = amp * (P0 * c - Q0 * s);
  Y0 = amp * (P0 * s + Q0 * c);
  // chi_1 = chi - pi/2: cos chi_1 = s, sin chi_1 = -c
  J1 = amp * (P1 * s + Q1 * c);
  Y1 = amp * (Q1 * s - P1 * c);
}

__device__ __forceinline__ void miller(double x, double& J0, double& Y0, double& J1,
                                       double& Y1) {
  const double tx = 2.0 / x;
  int N = (int)x + 36;
  N += N & 1;                 // even start index
  double jk1 = 0.0;           // J_(k+1)
  double jk = 1e-30;          // J_k, k = N
  double even = 0.0;          // sum_{m>=1} J_2m
  double sy0 = 0.0;           // sum_{m>=1} (-1)^m J_2m / m
  double sy1 = 0.0;           // sum_{m>=1} (-1)^m (J_(2m-1) - J_(2m+1)) / m
  double j1 = 0.0;
  // index N itself: even, m = N/2
  {
    const int m = N / 2;
    const double sg = (m & 1) ? -1.0 : 1.0;
    even += jk;
    sy0 += sg * jk * kInvM[m];
  }
  for (int k = N; k >= 1; --k) {
    const double jm = fma(k * tx, jk, -jk1);  // J_(k-1)
    const int o = k - 1;
    if (o >= 2 && !(o & 1)) {
      const int m = o / 2;
      const double sg = (m & 1) ? -1.0 : 1.0;
      even += jm;
      sy0 += sg * jm * kInvM[m];
    } else if (o & 1) {
      // odd index o enters (J_(2m-1) - J_(2m+1)) / m as +J_o with m = (o+1)/2
      // and as -J_o with m = (o-1)/2
      const int mp = (o + 1) / 2;
      if (mp <= N / 2 - 1) sy1 += ((mp & 1) ? -1.0 : 1.0) * jm * kInvM[mp];
      const int mm = (o - 1) / 2;
      if (mm >= 1 && mm <= N / 2 - 1) sy1 -= ((mm & 1) ? -1.0 : 1.0) * jm * kInvM[mm];
      if (o == 1) j1 = jm;
    }
    jk1 = jk;
    jk = jm;
    if (fabs(jk) > 1e200) {  // rescale to stay in range for small x
      jk *= 1e-200;
      jk1 *= 1e-200;
      even *= 1e-200;
      sy0 *= 1e-200;
      sy1 *= 1e-200;
      j1 *= 1e-200;
    }
  }
  const double inv = 1.0 / (jk + 2.0 * even);  // jk = J_0 (unnormalised)
  J0 = jk * inv;
  J1 = j1 * inv;
  const double lg = log(0.5 * x) + kGamma;
  Y0 = kTwoOverPi * (lg * J0 - 2.0 * sy0 * inv);
  Y1 = kTwoOverPi * (lg * J1 - J0 / x + sy1 * inv);
}

// x > 0
__device__ __forceinline__ void bessel01(double x, double& J0, double& Y0, double& J1,
                                         double& Y1) {
  if (x >= 20.0)
    asymptotic(x, J0, Y0, J1, Y1);
  else
    miller(x, J0, Y0, J1, Y1);
}

}  // namespace h64

// Nystrom entries of one off-diagonal pair (i != j) in FP64, r = |z_i - z_j|,
// (dx, dy) = z_i - z_j, w = Kress table entry w_{(i-j) mod n}, h = 2 pi / n.
//   soft:  a = h K + w K1 for K = L - i eta M (eq. 1)
//   hard:  a = S_ij = h M + w M1, b = D'_ij = h L' + w L'1 (eq. 2)
template <int BC>
__device__ __forceinline__ void pair_entries_fp64(double dx, double dy, double omega, double eta,
                                                  double h, double w, double nxj, double nyj,
                                                  double sj, double nxi, double nyi, double si,
                                                  double2& a, double2& b) {
  constexpr double inv4pi = 0.07957747154594767;  // 1 / (4 pi)
  const double r = sqrt(dx * dx + dy * dy);
  double J0, Y0, J1, Y1;
  h64::bessel01(omega * r, J0, Y0, J1, Y1);
  if constexpr (BC == 0) {
    const double c = (dx * nxj + dy * nyj) / r;
    a.x = 0.25 * h * (eta * sj * J0 - omega * c * Y1) - w * inv4pi * omega * c * J1;
    a.y = 0.25 * h * (omega * c * J1 + eta * sj * Y0) + w * inv4pi * eta * sj * J0;
    b = make_double2(0.0, 0.0);
  } else {
    a.x = -0.25 * h * Y0 * sj - w * inv4pi * J0 * sj;
    a.y = 0.25 * h * J0 * sj;
    const double cp = -(dx * nxi + dy * nyi) / r * sj / si;
    b.x = -0.25 * h * omega * cp * Y1 - w * inv4pi * omega * J1 * cp;
    b.y = 0.25 * h * omega * cp * J1;
  }
}
