// FP32 evaluation of one Nystrom entry pair with omega r >= kX0 (shared by the
// fused matrix-free matvec and the stored-matrix assembly).  See the header
// comment of matvec_fp32.cu for the two-float phase and the asymptotic
// Hankel expansion (A&S 9.2.5, 9.2.9, 9.2.10).
#pragma once

// FP32 geometry of an operator: hi/lo coordinates, unnormalised normal, speed.
// Stored in one buffer of 11 n floats: xh, xl, yh, yl, nx, ny, sp, w32 (Kress
// table), c32 (spectral-derivative circulant), and the Kress table twice over
// (2 n floats, entry i - j + n holds w_{(i - j) mod n}).
struct geo32 {
  float *xh, *xl, *yh, *yl, *nx, *ny, *sp;
};

// packed per-node copies for the fused kernels, after the 11 n floats above:
// float4 (x hi, x lo, y hi, y lo) and float4 (nu1, nu2, |z'|, 0), n of each,
// starting on a 16-byte boundary
inline size_t geo32_pack_offset(int n) { return ((size_t)11 * n + 3) & ~size_t(3); }
inline size_t geo32_floats(int n) { return geo32_pack_offset(n) + (size_t)8 * n; }

inline geo32 geo32_at(float* base, int n) {
  return geo32{base, base + n, base + 2 * n, base + 3 * n, base + 4 * n, base + 5 * n,
               base + 6 * n};
}

// omega = wh + wl (two-float), winv ~ 1/omega, eta, h = 2 pi / n
struct omega32 {
  float wh, wl, winv, eta, h;
};

constexpr float kX0 = 16.0f;  // asymptotic expansion used for omega r >= kX0

// Cody-Waite split of 2 pi: C1 has 10 significant bits
constexpr float kC1 = 6.28125f;
constexpr float kC2 = 0.0019353071693331003f;
constexpr float kC3 = 1.0253131677018246e-11f;
constexpr float kPi4H = 0.7853981852531433f;
constexpr float kPi4L = -2.1855695031547384e-08f;
constexpr float kInv2Pi = 0.15915493667125702f;
constexpr float kSqrt2OverPi = 0.7978845834732056f;
constexpr float kInv4Pi = 0.07957747154594767f;

// two-float helpers --------------------------------------------------------
__device__ __forceinline__ void two_diff(float a, float b, float& s, float& e) {
  s = a - b;
  const float v = s - a;
  e = (a - (s - v)) - (b + v);
}

// Entries of one pair with omega r >= kX0 (outside the band).
// (xh, xl, yh, yl) of target i and source j; returns soft a, hard (a = S, b = D').
template <int BC>
__device__ __forceinline__ void pair_entries_fp32(const omega32& P, float txh, float txl,
                                                  float tyh, float tyl, float tnx, float tny,
                                                  float tsp, float sxh, float sxl, float syh,
                                                  float syl, float snx, float sny, float ssp,
                                                  float w, float2& a, float2& b) {
  float dxs, dxe, dys, dye;
  two_diff(txh, sxh, dxs, dxe);
  dxe += txl - sxl;
  two_diff(tyh, syh, dys, dye);
  dye += tyl - syl;
  // r^2 = (dxs + dxe)^2 + (dys + dye)^2 as two-float
  const float px = dxs * dxs, qx = fmaf(dxs, dxs, -px);
  const float py = dys * dys, qy = fmaf(dys, dys, -py);
  const float t = px + py;
  const float tv = t - px;
  const float te = (px - (t - tv)) + (py - tv);
  const float lo = te + qx + qy + 2.0f * fmaf(dxs, dxe, dys * dye);
  const float r2 = t + lo;
  const float r2l = lo - (r2 - t);
  const float rinv = rsqrtf(r2);
  const float rh = r2 * rinv;
  const float rl = (fmaf(-rh, rh, r2) + r2l) * (0.5f * rinv);
  // x = omega r as two-float
  const float xh = P.wh * rh;
  const float xl = fmaf(P.wh, rh, -xh) + fmaf(P.wh, rl, P.wl * rh);
  // chi = x - pi/4 reduced to [-pi, pi]
  const float k = rintf(fmaf(xh, kInv2Pi, -0.125f));
  float chi = fmaf(-k, kC1, xh);
  chi = fmaf(-k, kC2, chi);
  chi = fmaf(-k, kC3, chi);
  chi = (chi - kPi4H) + (xl - kPi4L);
  float s, c;
  __sincosf(chi, &s, &c);
  // Hankel asymptotic expansion, t = 1/x
  const float ti = rinv * P.winv;
  const float t2 = ti * ti;
  const float P0 = fmaf(t2, fmaf(t2, fmaf(t2, -0.5725014209747314f, 0.112152099609375f), -0.0703125f), 1.0f);
  const float Q0 = ti * fmaf(t2, fmaf(t2, fmaf(t2, 1.7277275025844574f, -0.22710800170898438f), 0.0732421875f), -0.125f);
  const float P1 = fmaf(t2, fmaf(t2, fmaf(t2, 0.6765925884246826f, -0.144195556640625f), 0.1171875f), 1.0f);
  const float Q1 = ti * fmaf(t2, fmaf(t2, fmaf(t2, -1.993531733751297f, 0.2775764465332031f), -0.1025390625f), 0.375f);
  const float amp = kSqrt2OverPi * rsqrtf(xh);
  const float J0 = amp * (P0 * c - Q0 * s);
  const float Y0 = amp * (P0 * s + Q0 * c);
  const float J1 = amp * (P1 * s + Q1 * c);
  const float Y1 = amp * (Q1 * s - P1 * c);
  const float dx = dxs + dxe, dy = dys + dye;
  const float omega = P.wh;
  const float hq = 0.25f * P.h;
  if constexpr (BC == 0) {
    const float cc = (dx * snx + dy * sny) * rinv;
    const float es = P.eta * ssp;
    const float oc = omega * cc;
    a.x = hq * (es * J0 - oc * Y1) - w * kInv4Pi * oc * J1;
    a.y = hq * (oc * J1 + es * Y0) + w * kInv4Pi * es * J0;
  } else {
    a.x = -hq * Y0 * ssp - w * kInv4Pi * J0 * ssp;
    a.y = hq * J0 * ssp;
    const float cp = -(dx * tnx + dy * tny) * rinv * ssp / tsp;
    const float oc = omega * cp;
    b.x = -hq * oc * Y1 - w * kInv4Pi * oc * J1;
    b.y = hq * oc * J1;
  }
}

