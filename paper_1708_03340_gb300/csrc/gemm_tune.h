// gemm_tune.h -- tile-shape table of the SIMT contraction kernel.
// Written by paper_1708_03340_gb300/tune_gemm.py from timings on GB300; change
// it by rerunning the tuner, not by hand.
#pragma once
namespace htgb {
constexpr int kTuneTallM = 256;          // items with M >= this are tall (and square if N >= it too)
constexpr double kTuneTallShare = 0.5;   // 128 x 64 tiles when tall items hold this share of a launch's flops
constexpr double kTuneSquareShare = 0.6; // 128 x 128 tiles (uncompensated launches) above this square share
constexpr int kTuneCompLen = 256;        // Kahan-compensated FP32 sums when a CTA adds more products (accuracy, not tuned)
}  // namespace htgb
