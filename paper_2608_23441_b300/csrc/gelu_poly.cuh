// Generated by paper_2608_23441_b300/gelu_fit.py; do not edit.
// R(a) = erfcx(a / sqrt 2) / 2 ~= sum_k gelu_r(k) a^k on [0, kGeluClamp] (R(0) = 1/2
// exact), the weighted minimax fit that bounds the error of
// GELU(x) = max(x, 0) - |x| exp(-x^2 / 2) R(|x|).
#pragma once

namespace ipfb {

constexpr int kGeluDeg = 11;
constexpr float kGeluClamp = 6.0f;
// coefficient k of R (a function, so that unrolled device loops fold it to an immediate)
constexpr float gelu_r(int k) {
  return
  k == 0 ? 0.5f :
  k == 1 ? -0.39893442392349243f :
  k == 2 ? 0.2499035894870758f :
  k == 3 ? -0.13251525163650513f :
  k == 4 ? 0.06128989905118942f :
  k == 5 ? -0.0246585663408041f :
  k == 6 ? 0.008352464996278286f :
  k == 7 ? -0.0022560488432645798f :
  k == 8 ? 0.0004543154500424862f :
  k == 9 ? -6.274333281908184e-05f :
  k == 10 ? 5.226916982792318e-06f :
  k == 11 ? -1.9617628765900008e-07f :
  0.0f;
}

}  // namespace ipfb
