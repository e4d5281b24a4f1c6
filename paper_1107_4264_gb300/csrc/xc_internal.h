// xc_internal.h -- definitions shared by the engine's host and device code.
#pragma once

#include <cmath>
#include <cstdint>

#if defined(__CUDACC__)
#define XC_HD __host__ __device__ __forceinline__
#else
#define XC_HD inline
#endif

namespace xc {

// Lower-triangle block map of Sec. 4.2: block (bx, by) with bx <= by has
// linear index g = by(by+1)/2 + bx.
XC_HD int64_t tri_index(int64_t bx, int64_t by) { return by * (by + 1) / 2 + bx; }

// Inverse of tri_index.  The paper evaluates b_y = floor(-1/2 + sqrt(1/4 + 2g))
// with the fast square root; the estimate is then corrected with exact integer
// comparisons so that rounding of the square root can never pick a wrong row.
XC_HD void tri_coords(int64_t g, int64_t* bx, int64_t* by) {
  int64_t y = (int64_t)floor(-0.5 + sqrt(0.25 + 2.0 * (double)g));
  while (y > 0 && y * (y + 1) / 2 > g) --y;
  while ((y + 1) * (y + 2) / 2 <= g) ++y;
  *by = y;
  *bx = g - y * (y + 1) / 2;
}

// Device status word bits.
enum : int { kStatusTimeout = 1, kStatusRange = 2 };

// Geometry of one engine (device-side copy of the handle's sizes).
struct Geometry {
  int N;        // stations
  int P;        // polarisations (1 or 2)
  int F;        // channels
  int T;        // samples per integration
  int R;        // real operand rows per channel = 2 * P * N
  int Tp;       // T rounded up to the operand K-block (64)
  int64_t NB;   // baselines = N(N+1)/2
};

}  // namespace xc
