// A colour-split field of element type T: the iterate (red, black), its ping-pong
// partner for the temporally blocked kernel, and the right-hand-side term of the update
// (h2*f for the FP64 solve; the scaled defect for the FP32 inner solve of the
// mixed-precision refinement).  Row pitch W elements, 256-byte aligned rows.
#pragma once

#include <cuda.h>

namespace rbgs {

template <typename T>
struct ColourField {
    int n = 0;
    int W = 0;                 // elements per colour row
    T *u[2] = {nullptr, nullptr};
    T *alt[2] = {nullptr, nullptr};
    T *hf[2] = {nullptr, nullptr};
    // tensor maps for the temporal kernel: [0..1] u, [2..3] alt, [4..5] hf
    CUtensorMap maps[6];
    bool maps_ready = false;
    int maps_box_w = 0, maps_box_h = 0;
};

// Elements per colour row for element size `bytes`: ceil((n+2)/2) rounded up to 256 B.
inline int colour_width_bytes(int n, int bytes) {
    const int per = 256 / bytes;
    const int w = (n + 3) / 2;
    return (w + per - 1) / per * per;
}

}  // namespace rbgs
