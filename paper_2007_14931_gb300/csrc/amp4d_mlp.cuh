// Shape and parameter layout of the learned-proposal MLP 4 -> 64 -> 64 -> 1
// (tanh hidden units, softplus output): W1[64][4], b1[64], W2[64][64] (row =
// output unit), b2[64], W3[64], b3.
#pragma once

namespace amp4d {

constexpr int MH = 64;
constexpr int MLP_P = MH * 4 + MH + MH * MH + MH + MH + 1;  // 4545
constexpr int OFF_B1 = MH * 4, OFF_W2 = OFF_B1 + MH, OFF_B2 = OFF_W2 + MH * MH;
constexpr int OFF_W3 = OFF_B2 + MH, OFF_B3 = OFF_W3 + MH;

// Points per CTA tile of the gradient kernel: each CTA writes one partial row of
// MLP_P + 1 floats, and a set of n points takes at most ceil(n / MLP_GRAD_TILE) CTAs.
constexpr int MLP_GRAD_TILE = 64;

}  // namespace amp4d
