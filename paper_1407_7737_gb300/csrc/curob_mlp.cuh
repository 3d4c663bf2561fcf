// curob_mlp.cuh -- the learned pre-screen: an MLP surrogate 100 -> 256 -> 256
// -> 1 (GELU) of one benchmark function, trained and run with BF16 operands
// and FP32 accumulation on the tensor cores.
//
// Model: u = x / 128; a1 = W1 u + b1, h1 = gelu(a1); a2 = W2 h1 + b2,
// h2 = gelu(a2); y = w3 . h2 + b3, gelu(a) = a Phi(a) (Hendrycks and Gimpel
// 2016).  y predicts (t - mu) / sd, t = log(f - f_opt + 1), mu and sd the
// mean and standard deviation of t over the training set; loss = mean squared
// error; optimiser AdamW (Loshchilov and Hutter 2019).
//
// Every layer, forward and backward, is one launch of mlp_gemm_kernel: a
// 128-row tile C = A B^T on tcgen05 (kind::f16, BF16 operands, FP32
// accumulators in TMEM), both operands K-major in global memory and brought
// into shared memory by TMA tensor copies with the 64-byte swizzle, with the
// layer's bias, activation, loss and back-propagation arithmetic fused into
// the epilogue that drains TMEM.
#pragma once

#include <cstdint>

#include "../../include/curob.h"

namespace curob {

constexpr int kSurIn = 100;     // input dimension
constexpr int kSurInPad = 128;  // K of the first layer, zero-padded
constexpr int kSurH = 256;      // hidden width
// Flat parameter vector: W1 (256 x 100, row = output), b1, W2 (256 x 256),
// b2, w3, b3.
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kSurH * kSurIn;
constexpr int kOffW2 = kOffB1 + kSurH;
constexpr int kOffB2 = kOffW2 + kSurH * kSurH;
constexpr int kOffW3 = kOffB2 + kSurH;
constexpr int kOffB3 = kOffW3 + kSurH;
constexpr int kSurParams = kOffB3 + 1;  // 91905

}  // namespace curob
