// Generated by rf_poly_fit.py: Chebyshev-interpolant coefficients
// (lowest degree first, in v = t - t0 with t = u^2 or x^2), rounded to binary32.
#pragma once

namespace fqpoly {

constexpr float kSincUMax = 5.0f;
constexpr float kTapXMax = 0.8f;
constexpr float kSincCentre = 12.5f;
// kSincPoly0 .. kSincPoly7
constexpr float kSincPoly0 = -1.085637435e-01f;
constexpr float kSincPoly1 = -3.259358928e-02f;
constexpr float kSincPoly2 = 3.041254589e-03f;
constexpr float kSincPoly3 = -9.410488565e-05f;
constexpr float kSincPoly4 = 1.518525664e-06f;
constexpr float kSincPoly5 = -1.523321025e-08f;
constexpr float kSincPoly6 = 1.053542184e-10f;
constexpr float kSincPoly7 = -5.274230488e-13f;
// kSinPoly0 .. kSinPoly3
constexpr float kSinPoly0 = 1.000000000e+00f;
constexpr float kSinPoly1 = -1.666664928e-01f;
constexpr float kSinPoly2 = 8.331936784e-03f;
constexpr float kSinPoly3 = -1.949134457e-04f;
// kCosPoly0 .. kCosPoly4
constexpr float kCosPoly0 = 1.000000000e+00f;
constexpr float kCosPoly1 = -5.000000000e-01f;
constexpr float kCosPoly2 = 4.166661203e-02f;
constexpr float kCosPoly3 = -1.388644567e-03f;
constexpr float kCosPoly4 = 2.436412797e-05f;

}  // namespace fqpoly
