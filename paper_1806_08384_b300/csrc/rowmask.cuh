// rowmask.cuh -- a 256-row chunk's selection mask in its two forms.
//
// Lane bytes: the interpreter leaves lane l of a warp an 8-bit mask whose bit
// i < 4 is row 4l + i of the chunk and bit 4 + i is row 128 + 4l + i; stored
// as one byte per lane, a chunk's mask is 32 bytes.  Row-order words: word k
// holds rows 32k .. 32k + 31, bit j for row 32k + j.  Ranking the selected
// rows of a chunk in row order works on the second form.
#pragma once
#include <stdint.h>

namespace sel {

// The low nibbles of the 4 bytes of x, packed into 16 bits.
__device__ __forceinline__ uint32_t pack_nibbles(uint32_t x) {
    x &= 0x0F0F0F0Fu;
    x = (x | (x >> 4)) & 0x00FF00FFu;
    return (x | (x >> 8)) & 0x0000FFFFu;
}

// Rewrites one chunk's 32 lane bytes (two uint4: x holds lanes 0..15, y lanes
// 16..31) as its 8 row-order words.
__device__ __forceinline__ void lane_bytes_to_rows(uint4* w4, const uint4& x, const uint4& y) {
    const uint32_t w[8] = {x.x, x.y, x.z, x.w, y.x, y.y, y.z, y.w};   // w[i]: lanes 4i .. 4i + 3
    uint32_t r[8];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        r[k] = pack_nibbles(w[2 * k]) | (pack_nibbles(w[2 * k + 1]) << 16);
        r[4 + k] = pack_nibbles(w[2 * k] >> 4) | (pack_nibbles(w[2 * k + 1] >> 4) << 16);
    }
    w4[0] = make_uint4(r[0], r[1], r[2], r[3]);
    w4[1] = make_uint4(r[4], r[5], r[6], r[7]);
}

// Position of the (o+1)-th set bit of w (o < popc(w)).
__device__ __forceinline__ uint32_t select_bit(uint32_t w, uint32_t o) {
    uint32_t pos = 0, c;
    c = __popc(w & 0xFFFFu); if (o >= c) { o -= c; pos += 16; w >>= 16; }
    c = __popc(w & 0xFFu);   if (o >= c) { o -= c; pos += 8;  w >>= 8; }
    c = __popc(w & 0xFu);    if (o >= c) { o -= c; pos += 4;  w >>= 4; }
    c = __popc(w & 0x3u);    if (o >= c) { o -= c; pos += 2;  w >>= 2; }
    if (o >= (w & 1u)) pos += 1;
    return pos;
}

}  // namespace sel
