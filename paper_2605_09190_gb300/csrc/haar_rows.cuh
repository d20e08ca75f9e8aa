// haar_rows.cuh -- the support of the 1-D Haar rows, shared by the host's
// dictionary check and the exact SIMT correlation.
#pragma once

namespace aqmp {

// Haar row r of side b (Section 2.1 Eq. (2)) as two halves on which it is
// constant: rows r >= 1 of scale 2^floor(log2 r) are +v on [s, s + h) and
// -v on [s + h, s + 2h), with 2h = b / scale and s = (r - scale) 2h; row 0
// is constant on the whole block, taken as its halves [0, b/2), [b/2, b).
__host__ __device__ __forceinline__ void haar_halves(int r, int b, int &s, int &h) {
    if (r == 0) {
        s = 0;
        h = b / 2;
        return;
    }
    int scale = 1;
    while (scale * 2 <= r) scale *= 2;
    h = b / scale / 2;
    s = (r - scale) * 2 * h;
}

}  // namespace aqmp
