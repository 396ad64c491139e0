// Coefficients of the logistic approximation of the standard normal CDF used by
// the tensor-core surrogate's GELU (GELU(z) = z Phi(z)):
//
//   Phi(z) ~ 1 / (1 + 2^(-z (C0 + C1 s + C2 s^2))),  s = min(z^2, Z2MAX),
//
// a weighted least-squares (minimax-like) fit of Phi on [-30, 30]; the clamp
// keeps the exponent monotone in z.  Maximum error 1.9e-5 in Phi and 5.5e-5 in
// GELU over that range (checked against erf in the CPU tests), well below the
// bfloat16 rounding that the activations get next.
//
// The kernel evaluates the same function through the hyperbolic tangent,
// 1 / (1 + 2^-x) = (1 + tanh(x ln2 / 2)) / 2, with the coefficients scaled by
// TANH_SCALE = ln 2 / 2 (rounded to float), so that each activation costs one special-function
// instruction instead of two (exp2 and reciprocal).
#pragma once

#define DFP2S_GELU_C0 0x1.269efep+1f
#define DFP2S_GELU_C1 0x1.b2e704p-4f
#define DFP2S_GELU_C2 -0x1.ddbf44p-11f
#define DFP2S_GELU_Z2MAX 25.0f
#define DFP2S_GELU_TANH_SCALE 0x1.62e430p-2f
