// FP32 evaluation of one Nystrom entry pair with omega r >= kX0 (shared by the
// fused matrix-free matvec and the stored-matrix assembly).  See the header
// comment of matvec_fp32.cu for the two-float phase and the asymptotic
// Hankel expansion (A&S 9.2.5, 9.2.9, 9.2.10).
#pragma once

// FP32 geometry of an operator: coordinates times omega as hi/lo pairs,
// unnormalised normal, speed.
// Stored in one buffer: 9 n floats xh, xl, yh, yl, nx, ny, sp, w32 (Kress
// table), c32 (spectral-derivative circulant); then, for the fused
// tensor-core kernel, starting on 16-byte boundaries:
//   n float4 coordinates      (omega x hi, lo, omega y hi, lo)
//   n float4 source factors   (omega hq c0 nu1, omega hq c0 nu2, hq c0 eta |z'|, hq c0 |z'|)
//   n float4 target factors   (omega nu1 / |z'|, omega nu2 / |z'|, 0, 0)
//   2 n + 8 float2: the Kress table twice over divided by pi h, entry
//   k = i - j + n holding the weights of sources j and j + 1,
//   (w_{k mod n}, w_{(k - 1) mod n}) / (pi h), then zeros
// with hq = h / 4 and c0 = sqrt(2 / pi) (nu = unnormalised normal, |z'| = speed).
struct geo32 {
  float *xh, *xl, *yh, *yl, *nx, *ny, *sp;
};

inline size_t geo32_pack_offset(int n) { return ((size_t)9 * n + 3) & ~size_t(3); }
inline size_t geo32_wk_offset(int n) { return geo32_pack_offset(n) + (size_t)12 * n; }
// (+ 128 floats of slack: the fused kernel copies whole 32-source tiles)
inline size_t geo32_floats(int n) { return geo32_wk_offset(n) + (size_t)4 * n + 16 + 128; }

inline geo32 geo32_at(float* base, int n) {
  return geo32{base, base + n, base + 2 * n, base + 3 * n, base + 4 * n, base + 5 * n,
               base + 6 * n};
}

// omega (FP32), eta, h = 2 pi / n: the operator constants of the generic
// entries (the phase comes from the omega-scaled coordinates)
struct omega32 {
  float wh, eta, h;
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

// Special-function-unit approximations without subnormal handling: their
// arguments here are >= 16 (square roots) or reduced phases, never subnormal
__device__ __forceinline__ float rsqrt_sfu(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ void sincos_sfu(float x, float* s, float* c) {
  asm("sin.approx.ftz.f32 %0, %1;" : "=f"(*s) : "f"(x));
  asm("cos.approx.ftz.f32 %0, %1;" : "=f"(*c) : "f"(x));
}

// Distance and phase of one pair with omega r >= kX0.  Coordinates are scaled
// by omega, so the distance of two nodes is the Hankel argument x = omega r
// itself, and split as hi + lo with the hi parts on a grid coarse enough that
// the difference of two of them and the sum of the two squared differences
// are exact in FP32 (geometry set-up).  Then x^2 = H + C with H = dxh^2 + dyh^2
// exact and the lo-part terms C = dxl (2 dxh + dxl) + dyl (2 dyh + dyl) in
// FP32; x^2 and x are carried as two-float numbers (error-free
// transformations built from fmaf), and chi = x - pi/4 is reduced modulo 2 pi
// with a three-part Cody-Waite constant.  Phase error ~2^(e - 33) rad when
// omega |z| < 2^e (6.5e-7 rad at most for the kite at omega = 2048).
struct pair_phase {
  float dx, dy;   // omega (z_i - z_j)
  float xinv;     // 1 / (omega r)
  float ra;       // (omega r)^(-1/2)
  float s, c;     // sin, cos of omega r - pi / 4
};

__device__ __forceinline__ pair_phase pair_phase32(float txh, float txl, float tyh, float tyl,
                                                   float sxh, float sxl, float syh, float syl) {
  pair_phase f;
  const float dxh = txh - sxh, dxl = txl - sxl;   // dxh, dyh exact
  const float dyh = tyh - syh, dyl = tyl - syl;
  const float H = fmaf(dxh, dxh, dyh * dyh);      // exact
  const float C = fmaf(dxl, fmaf(2.0f, dxh, dxl), dyl * fmaf(2.0f, dyh, dyl));
  // x^2 = H + C as two-float (TwoSum)
  const float x2 = H + C;
  const float bv = x2 - H;
  const float x2l = (H - (x2 - bv)) + (C - bv);
  const float xinv = rsqrt_sfu(x2);
  const float xh = x2 * xinv;
  // x lo, less the lo part of the pi/4 split
  const float xl4 = fmaf(fmaf(-xh, xh, x2) + x2l, 0.5f * xinv, -kPi4L);
  // chi = x - pi/4 reduced to [-pi, pi]
  const float k = rintf(fmaf(xh, kInv2Pi, -0.125f));
  float chi = fmaf(-k, kC1, xh);
  chi = fmaf(-k, kC2, chi);
  chi = fmaf(-k, kC3, chi - kPi4H) + xl4;
  sincos_sfu(chi, &f.s, &f.c);
  f.dx = dxh + dxl;
  f.dy = dyh + dyl;
  f.xinv = xinv;
  f.ra = rsqrt_sfu(xh);
  return f;
}

// The same distance and phase to the accuracy of the fused tensor-core
// kernel, whose entries reach the tensor cores as bf16 hi + lo pairs (2^-17
// relative): the lo part of x comes from H - xh^2 (one fma, of the size of C)
// plus C instead of from the exact sum H + C, the Cody-Waite constant has two
// parts (the third, k C3, is 1.6e-12 omega r rad) and the lo part of pi/4 is
// dropped (2.2e-8 rad).  Phase error a few 1e-7 rad for the kite at
// omega = 2048.
__device__ __forceinline__ pair_phase pair_phase32_tc(float txh, float txl, float tyh, float tyl,
                                                      float sxh, float sxl, float syh, float syl) {
  pair_phase f;
  const float dxh = txh - sxh, dxl = txl - sxl;   // dxh, dyh exact
  const float dyh = tyh - syh, dyl = tyl - syl;
  const float H = fmaf(dxh, dxh, dyh * dyh);      // exact
  const float C = fmaf(dxl, fmaf(2.0f, dxh, dxl), dyl * fmaf(2.0f, dyh, dyl));
  const float x2 = H + C;
  const float xinv = rsqrt_sfu(x2);
  const float xh = x2 * xinv;
  const float xl = (fmaf(-xh, xh, H) + C) * (0.5f * xinv);
  const float k = rintf(fmaf(xh, kInv2Pi, -0.125f));
  float chi = fmaf(-k, kC1, xh);                  // exact
  chi = fmaf(-k, kC2, chi);
  chi = (chi - kPi4H) + xl;
  sincos_sfu(chi, &f.s, &f.c);
  f.dx = dxh + dxl;
  f.dy = dyh + dyl;
  f.xinv = xinv;
  f.ra = rsqrt_sfu(xh);
  return f;
}

// Hankel's asymptotic expansion for x >= kX0 (t = 1/x), three terms of each
// of P and Q (A&S 9.2.9, 9.2.10), without the common factor c0 x^(-1/2):
// J_m = c0 ra j_m, Y_m = c0 ra y_m.  The remainder is below the first omitted
// term (A&S 9.2.10 remark), < 4.1e-8 for x >= 16: under one FP32 ulp.
__device__ __forceinline__ void hankel_asym32(float ti, float s, float c, float& j0, float& y0,
                                              float& j1, float& y1) {
  const float t2 = ti * ti;
  const float P0 = fmaf(t2, fmaf(t2, 0.112152099609375f, -0.0703125f), 1.0f);
  const float Q0 = ti * fmaf(t2, fmaf(t2, -0.22710800170898438f, 0.0732421875f), -0.125f);
  const float P1 = fmaf(t2, fmaf(t2, -0.144195556640625f, 0.1171875f), 1.0f);
  const float Q1 = ti * fmaf(t2, fmaf(t2, 0.2775764465332031f, -0.1025390625f), 0.375f);
  j0 = fmaf(P0, c, -Q0 * s);
  y0 = fmaf(P0, s, Q0 * c);
  j1 = fmaf(P1, s, Q1 * c);
  y1 = fmaf(Q1, s, -P1 * c);
}

// Two terms of each of P and Q (the fused tensor-core kernel): the remainder
// is below the first omitted term, < 2.2e-6 relative for x >= 16 and
// < 1.4e-8 for x >= 64, near the bf16 hi + lo split's 2^-17.
__device__ __forceinline__ void hankel_asym32_tc(float ti, float s, float c, float& j0, float& y0,
                                                 float& j1, float& y1) {
  const float t2 = ti * ti;
  const float P0 = fmaf(t2, -0.0703125f, 1.0f);
  const float Q0 = ti * fmaf(t2, 0.0732421875f, -0.125f);
  const float P1 = fmaf(t2, 0.1171875f, 1.0f);
  const float Q1 = ti * fmaf(t2, -0.1025390625f, 0.375f);
  j0 = fmaf(P0, c, -Q0 * s);
  y0 = fmaf(P0, s, Q0 * c);
  j1 = fmaf(P1, s, Q1 * c);
  y1 = fmaf(Q1, s, -P1 * c);
}

// Entries of one pair with omega r >= kX0 (outside the band).
// (xh, xl, yh, yl) of target i and source j; returns soft a, hard (a = S, b = D').
template <int BC>
__device__ __forceinline__ void pair_entries_fp32(const omega32& P, float txh, float txl,
                                                  float tyh, float tyl, float tnx, float tny,
                                                  float tsp, float sxh, float sxl, float syh,
                                                  float syl, float snx, float sny, float ssp,
                                                  float w, float2& a, float2& b) {
  const pair_phase f = pair_phase32(txh, txl, tyh, tyl, sxh, sxl, syh, syl);
  float j0, y0, j1, y1;
  hankel_asym32(f.xinv, f.s, f.c, j0, y0, j1, y1);
  const float amp = kSqrt2OverPi * f.ra;
  const float J0 = amp * j0, Y0 = amp * y0, J1 = amp * j1, Y1 = amp * y1;
  const float omega = P.wh;
  const float hq = 0.25f * P.h;
  if constexpr (BC == 0) {
    const float cc = (f.dx * snx + f.dy * sny) * f.xinv;
    const float es = P.eta * ssp;
    const float oc = omega * cc;
    a.x = hq * (es * J0 - oc * Y1) - w * kInv4Pi * oc * J1;
    a.y = hq * (oc * J1 + es * Y0) + w * kInv4Pi * es * J0;
  } else {
    a.x = -hq * Y0 * ssp - w * kInv4Pi * J0 * ssp;
    a.y = hq * J0 * ssp;
    const float cp = -(f.dx * tnx + f.dy * tny) * f.xinv * ssp / tsp;
    const float oc = omega * cp;
    b.x = -hq * oc * Y1 - w * kInv4Pi * oc * J1;
    b.y = hq * oc * J1;
  }
}

// Entry kinds: the sound-soft combination of eq. 1, or one of the two layer
// operators S, D' of the sound-hard operator of eq. 2
enum { KIND_SOFT = 0, KIND_S = 1, KIND_DP = 2 };

// The same entries with the per-node factors folded in, to the fused
// tensor-core kernel's accuracy (phase and series above): tg, sc = target and
// source coordinates, tq = target factors (D'
// only), sq = source factors, wk = Kress weight / (pi h); see the packed
// layout above.  With A = sq ra and B = omega hq c0 (nu_j . (z_i - z_j)) ra / r,
//   soft:  re = A j0 - B (y1 + wk j1),      im = B j1 + A (y0 + wk j0)
//   S:     re = -A' (y0 + wk j0),            im = A' j0        (A' = hq c0 |z'_j| ra)
//   D':    re = D (y1 + wk j1),              im = -D j1
// with D = omega (nu_i . (z_i - z_j)) / |z'_i| hq c0 |z'_j| ra / r.
template <int KIND>
__device__ __forceinline__ float2 entry_finish32(const pair_phase& f, float4 tq, float4 sq,
                                                 float wk) {
  float j0, y0, j1, y1;
  hankel_asym32_tc(f.xinv, f.s, f.c, j0, y0, j1, y1);
  float2 a;
  if constexpr (KIND == KIND_SOFT) {
    const float A = sq.z * f.ra;
    const float B = fmaf(f.dx, sq.x, f.dy * sq.y) * (f.xinv * f.ra);
    a.x = fmaf(A, j0, -B * fmaf(wk, j1, y1));
    a.y = fmaf(B, j1, A * fmaf(wk, j0, y0));
  } else if constexpr (KIND == KIND_S) {
    const float A = sq.w * f.ra;
    a.x = -A * fmaf(wk, j0, y0);
    a.y = A * j0;
  } else {
    const float D = fmaf(f.dx, tq.x, f.dy * tq.y) * (f.xinv * f.ra) * sq.w;
    a.x = D * fmaf(wk, j1, y1);
    a.y = -D * j1;
  }
  return a;
}

template <int KIND>
__device__ __forceinline__ float2 entry_folded32(float4 tg, float4 tq, float4 sc, float4 sq,
                                                 float wk) {
  return entry_finish32<KIND>(pair_phase32_tc(tg.x, tg.y, tg.z, tg.w, sc.x, sc.y, sc.z, sc.w), tq,
                              sq, wk);
}
