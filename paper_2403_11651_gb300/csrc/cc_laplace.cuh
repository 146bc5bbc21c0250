// Rate of one latent under the Laplace model of the ARM output (eq. (1)), shared by the
// ARM kernels.
#pragma once

namespace cc {

struct LapOut {
  float bits, g_y, g_mu, g_s;  // bits and its derivatives wrt y_hat, mu, s
};

// -log2 P(y_hat) for the Laplace law (mu, b = exp(clamp(s))), P floored at 2^-16.
// With d = y_hat - mu: for |d| >= 1/2 both bin edges lie on one side of mu and
//   P = 1/2 exp(-(|d| - 1/2)/b) (1 - exp(-1/b));
// otherwise P = 1 - 1/2 (exp(-(1/2 + d)/b) + exp(-(1/2 - d)/b)), formed with expm1 so
// nothing cancels.  Derivatives of ln P:
//   outer: d/dd = -sign(d)/b,  d/ds = ((|d| - 1/2) - 1/expm1(1/b)) / b
//   inner: d/dd = (e1 - e2) / (2 b P),  d/ds = -(e1 (1/2 + d) + e2 (1/2 - d)) / (2 b P)
__device__ __forceinline__ LapOut laplace_bits(float yh, float mu, float s) {
  constexpr float kLogBMin = -4.60517018598809136f;  // ln 1e-2
  constexpr float kLogBMax = 6.90775527898213705f;   // ln 1e3
  constexpr float kInvLn2 = 1.44269504088896341f;
  constexpr float kPMin = 1.52587890625e-05f;        // 2^-16
  const float sc = fminf(fmaxf(s, kLogBMin), kLogBMax);
  const float b = expf(sc);
  const float ib = 1.0f / b;
  const float d = yh - mu;
  const float ad = fabsf(d);
  float P, gd, gs;
  if (ad >= 0.5f) {
    P = 0.5f * expf(-(ad - 0.5f) * ib) * (-expm1f(-ib));
    gd = -copysignf(ib, d);
    gs = ((ad - 0.5f) - 1.0f / expm1f(ib)) * ib;
  } else {
    const float a1 = (0.5f + d) * ib, a2 = (0.5f - d) * ib;
    const float e1 = expf(-a1), e2 = expf(-a2);
    P = -0.5f * (expm1f(-a1) + expm1f(-a2));
    const float iP = 1.0f / P;
    gd = 0.5f * (e1 - e2) * ib * iP;
    gs = -0.5f * (e1 * a1 + e2 * a2) * iP;
  }
  LapOut o;
  if (!(P >= kPMin)) {
    o.bits = 16.0f;
    o.g_y = o.g_mu = o.g_s = 0.0f;
    return o;
  }
  o.bits = -log2f(P);
  o.g_y = -gd * kInvLn2;
  o.g_mu = gd * kInvLn2;
  o.g_s = (s >= kLogBMin && s <= kLogBMax) ? -gs * kInvLn2 : 0.0f;
  return o;
}

}  // namespace cc
