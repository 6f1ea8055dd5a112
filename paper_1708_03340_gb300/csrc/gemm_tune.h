// gemm_tune.h -- tile-shape table of the SIMT contraction kernel.
// Written by paper_1708_03340_gb300/tune_gemm.py from timings on GB300; edit
// by rerunning the tuner, not by hand.
#pragma once
namespace htgb {
constexpr int kTuneTallM = 128;        // items with M >= this ...
constexpr int kTuneTallMinN = 1;       // ... and N >= this count as tall
constexpr double kTuneTallShare = 0.5;  // 128 x 64 tiles when tall items hold this share of the flops
constexpr int kTuneCompLen = 256;      // Kahan-compensated FP32 sums when a CTA adds more products
}  // namespace htgb
