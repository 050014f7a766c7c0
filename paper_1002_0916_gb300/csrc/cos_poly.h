// cos_poly.h -- written by gen_cos_poly.py; do not edit.
// cos(d) ~= sum_k COS_Ck (d^2)^k for d in [0, pi] (Lawson minimax fit,
// degree 6 in d^2; max error in FP32 evaluation 6.15e-07).
#pragma once

namespace cgh {

constexpr float COS_C0 = 1.0f;
constexpr float COS_C1 = -0.49999991059303284f;
constexpr float COS_C2 = 0.04166649281978607f;
constexpr float COS_C3 = -0.001388781820423901f;
constexpr float COS_C4 = 2.477006273693405e-05f;
constexpr float COS_C5 = -2.707994326556218e-07f;
constexpr float COS_C6 = 1.7246171157836443e-09f;

}  // namespace cgh
