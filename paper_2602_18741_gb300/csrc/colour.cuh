// CIELAB and colour-difference formulas shared by the metrics kernels.
#pragma once

#include "common.cuh"

namespace hsc {

__device__ __forceinline__ float lab_f(float t) {
  const float d = 6.0f / 29.0f;
  return (t > d * d * d) ? cbrtf(t) : t / (3.0f * d * d) + 4.0f / 29.0f;
}

__device__ __forceinline__ void to_lab(float X, float Y, float Z, const float* w, float& L, float& a, float& b) {
  const float fx = lab_f(X / w[0]), fy = lab_f(Y / w[1]), fz = lab_f(Z / w[2]);
  L = 116.0f * fy - 16.0f;
  a = 500.0f * (fx - fy);
  b = 200.0f * (fy - fz);
}

constexpr float kDeg = 57.29577951308232f;
constexpr float kRad = 0.017453292519943295f;

__device__ __forceinline__ float pow7(float x) {
  const float x2 = x * x;
  return x2 * x2 * x2 * x;
}

// CIEDE2000 (CIE 142-2001), kL = kC = kH = 1; colour 1 is the reference.
__device__ __forceinline__ float de2000(float L1, float a1, float b1, float L2, float a2, float b2) {
  const float C1 = sqrtf(a1 * a1 + b1 * b1), C2 = sqrtf(a2 * a2 + b2 * b2);
  const float Cm7 = pow7(0.5f * (C1 + C2));
  const float G = 0.5f * (1.0f - sqrtf(Cm7 / (Cm7 + 6103515625.0f)));  // 25^7
  const float ap1 = (1.0f + G) * a1, ap2 = (1.0f + G) * a2;
  const float Cp1 = sqrtf(ap1 * ap1 + b1 * b1), Cp2 = sqrtf(ap2 * ap2 + b2 * b2);
  float h1 = (ap1 == 0.0f && b1 == 0.0f) ? 0.0f : atan2f(b1, ap1) * kDeg;
  float h2 = (ap2 == 0.0f && b2 == 0.0f) ? 0.0f : atan2f(b2, ap2) * kDeg;
  if (h1 < 0.0f) h1 += 360.0f;
  if (h2 < 0.0f) h2 += 360.0f;
  const float dL = L2 - L1, dC = Cp2 - Cp1;
  const float pc = Cp1 * Cp2;
  float dh = h2 - h1;
  if (pc == 0.0f) dh = 0.0f;
  else if (dh > 180.0f) dh -= 360.0f;
  else if (dh < -180.0f) dh += 360.0f;
  const float dH = 2.0f * sqrtf(pc) * sinf(0.5f * dh * kRad);
  const float Lm = 0.5f * (L1 + L2), Cm = 0.5f * (Cp1 + Cp2);
  float hm = h1 + h2;
  if (pc != 0.0f) {
    if (fabsf(h1 - h2) <= 180.0f) hm *= 0.5f;
    else if (hm < 360.0f) hm = 0.5f * (hm + 360.0f);
    else hm = 0.5f * (hm - 360.0f);
  }
  const float T = 1.0f - 0.17f * cosf((hm - 30.0f) * kRad) + 0.24f * cosf(2.0f * hm * kRad) +
                  0.32f * cosf((3.0f * hm + 6.0f) * kRad) - 0.20f * cosf((4.0f * hm - 63.0f) * kRad);
  const float e = (hm - 275.0f) / 25.0f;
  const float dtheta = 30.0f * expf(-e * e);
  const float Cm7b = pow7(Cm);
  const float RC = 2.0f * sqrtf(Cm7b / (Cm7b + 6103515625.0f));
  const float l50 = (Lm - 50.0f) * (Lm - 50.0f);
  const float SL = 1.0f + 0.015f * l50 / sqrtf(20.0f + l50);
  const float SC = 1.0f + 0.045f * Cm;
  const float SH = 1.0f + 0.015f * Cm * T;
  const float RT = -sinf(2.0f * dtheta * kRad) * RC;
  const float tL = dL / SL, tC = dC / SC, tH = dH / SH;
  return sqrtf(fmaxf(tL * tL + tC * tC + tH * tH + RT * tC * tH, 0.0f));
}

// CIE94, graphic arts (kL = 1, K1 = 0.045, K2 = 0.015); colour 1 is the reference.
__device__ __forceinline__ float de94(float L1, float a1, float b1, float L2, float a2, float b2) {
  const float C1 = sqrtf(a1 * a1 + b1 * b1), C2 = sqrtf(a2 * a2 + b2 * b2);
  const float dL = L1 - L2, dC = C1 - C2, da = a1 - a2, db = b1 - b2;
  const float dH2 = fmaxf(da * da + db * db - dC * dC, 0.0f);
  const float SC = 1.0f + 0.045f * C1, SH = 1.0f + 0.015f * C1;
  return sqrtf(dL * dL + (dC / SC) * (dC / SC) + dH2 / (SH * SH));
}


// CIE 1976 L*a*b* of XYZ relative to a white given per call.
__device__ __forceinline__ void to_lab_white(float X, float Y, float Z, float wx, float wy, float wz, float& L,
                                             float& a, float& b) {
  const float fx = lab_f(X / wx), fy = lab_f(Y / wy), fz = lab_f(Z / wz);
  L = 116.0f * fy - 16.0f;
  a = 500.0f * (fx - fy);
  b = 200.0f * (fy - fz);
}

}  // namespace hsc
