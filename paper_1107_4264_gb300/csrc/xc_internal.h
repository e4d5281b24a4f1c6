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

// Work items of the CTA-pair engine: the nib(nib+1)/2 lower blocks (r, c),
// r >= c, of a channel with nib block rows, two per item, both sharing
// their column block.  In column c the rows c, c+1, ... pair off from the
// diagonal down (floor((nib-c)/2) items).  A column with an odd count leaves
// its last block (nib-1, c); that block is taken transposed, as rows c times
// columns nib-1 (the mirror block), so the leftovers of the columns
// c = nib-1, nib-3, ... all have column block nib-1 and pair among
// themselves, the very last one alone when their count is odd.
XC_HD int pair_items(int nib) {
  const int L = (nib + 1) / 2;  // leftovers
  return nib * nib / 4 + (L + 1) / 2;
}

// Item i (0 <= i < pair_items(nib)): row blocks a0, a1 of the pair's two
// CTAs and their common column block b.  a_k < b marks a transposed block;
// *single is set when the item holds one block only (a1 repeats a0 and the
// second CTA's result is discarded).
XC_HD void pair_coords(int i, int nib, int* a0, int* a1, int* b, int* single) {
  for (int c = 0; c < nib; ++c) {
    const int m = (nib - c) / 2;
    if (i < m) {
      *a0 = c + 2 * i;
      *a1 = *a0 + 1;
      *b = c;
      *single = 0;
      return;
    }
    i -= m;
  }
  const int L = (nib + 1) / 2;
  const int k0 = 2 * i, k1 = k0 + 1;
  *b = nib - 1;
  *a0 = nib - 1 - 2 * k0;
  *single = k1 >= L ? 1 : 0;
  *a1 = *single ? *a0 : nib - 1 - 2 * k1;
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
