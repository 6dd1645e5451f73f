// tiles.h -- tile shapes of the FP32 and BF16 step kernels, shared by their
// round-to-nearest and stochastic-rounding translation units.
#pragma once

// tile of the FP32 kernel: SPFM_F32_TX threads of 4 cells in x, SPFM_F32_TY rows
#ifndef SPFM_F32_TX
#define SPFM_F32_TX 16
#endif
#ifndef SPFM_F32_TY
#define SPFM_F32_TY 16
#endif

namespace spfm {
// the square tile of FP32 batch items of shape 1: 8 threads of 4 cells, 32 rows
// (32 x 32 cells, the same 128 consumer threads), for grids narrower than the
// 64-cell tile or whose x extent it would pad
constexpr int kSqTX = 8, kSqTY = 32;
// the BF16 tile: 8 threads of 8 cells in x, 16 rows
constexpr int kBfTX = 8, kBfTY = 16;
}  // namespace spfm
