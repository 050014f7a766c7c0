// cos_poly.h -- written by gen_cos_poly.py; do not edit.
// cos(d) ~= sum_k C_k (d^2)^k for d in [0, pi] (Lawson minimax fits):
// COS_C: degree 6 in d^2, max error in FP32 evaluation 6.15e-07;
// COS5_C: degree 5 in d^2, max error in FP32 evaluation 1.27e-06;
// sin(d) ~= d * sum_k S_k (d^2)^k for d in [0, pi]:
// SIN5_C: degree 5 in d^2, max error in FP32 evaluation 4.44e-07.
#pragma once

namespace cgh {

constexpr float COS_C0 = 1.0f;
constexpr float COS_C1 = -0.49999991059303284f;
constexpr float COS_C2 = 0.04166649281978607f;
constexpr float COS_C3 = -0.001388781820423901f;
constexpr float COS_C4 = 2.477006273693405e-05f;
constexpr float COS_C5 = -2.707994326556218e-07f;
constexpr float COS_C6 = 1.7246171157836443e-09f;

constexpr float COS5_C0 = 0.9999993443489075f;
constexpr float COS5_C1 = -0.49999457597732544f;
constexpr float COS5_C2 = 0.04165996238589287f;
constexpr float COS5_C3 = -0.0013859154423698783f;
constexpr float COS5_C4 = 2.420584496576339e-05f;
constexpr float COS5_C5 = -2.1980551423439465e-07f;

constexpr float SIN5_C0 = 0.9999996423721313f;
constexpr float SIN5_C1 = -0.16666558384895325f;
constexpr float SIN5_C2 = 0.008332425728440285f;
constexpr float SIN5_C3 = -0.00019809025980066508f;
constexpr float SIN5_C4 = 2.700008735700976e-06f;
constexpr float SIN5_C5 = -2.037002744259553e-08f;

}  // namespace cgh
