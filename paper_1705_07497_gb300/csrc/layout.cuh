// Internal image layout and the band geometry of the A^T storage.
//
// Image vectors inside the library are stored by 16 x 16 tiles (tiles in
// row-major order), each tile by 4 x 4 micro-tiles (row-major), each
// micro-tile row-major.  A micro-tile of double-float values is one 128-byte
// line, so the pixels a ray crosses in a short run lie in a few lines
// whatever the ray's direction.  The padded size is (ceil(N/16) * 16)^2;
// padding pixels belong to no ray and stay zero.
//
// A^T is stored by image tiles: for tile T and kept angle k, the bins whose
// rays can cross T form a contiguous band [band_lo(T, k), band_lo(T, k) + W_k)
// with W_k = floor(16 (|cos| + |sin|)) + 2 <= kBandMax bins (the tile's
// projection is 16 (|cos| + |sin|) detector units long), and an entry of A^T
// for a pixel of T is addressed by its local band index
// off_k + (b - band_lo(T, k)) (16 bits), off_k = W_0 + ... + W_{k-1}.  A
// tile's band of the sinogram is staged in shared memory once and then read
// per entry.
#pragma once

#include <cstdint>

namespace ct {

constexpr int kTile = 16;        // pixels per tile side
constexpr int kTilePix = 256;    // pixels per tile
constexpr int kBandMax = 32;     // bound on the bins of one (tile, angle) band (<= 24 are used)
constexpr int kBandChunkSlots = 3968;  // slots of a staged band chunk (31 KB in double-float)

__host__ __device__ inline int tiles_per_side(int n) { return (n + kTile - 1) / kTile; }

__host__ __device__ inline int64_t padded_pixels(int n)
{
    const int64_t t = tiles_per_side(n);
    return t * t * kTilePix;
}

// Internal index of pixel (i, j).
__host__ __device__ inline int64_t tiled_index(int i, int j, int tn)
{
    const int ti = i >> 4, tj = j >> 4, r = i & 15, c = j & 15;
    const int micro = ((r >> 2) << 6) | ((c >> 2) << 4) | ((r & 3) << 2) | (c & 3);
    return ((int64_t)(ti * tn + tj) << 8) | micro;
}

// Pixel (i, j) of an internal index.
__host__ __device__ inline void tiled_coords(int64_t t, int tn, int& i, int& j)
{
    const int tile = (int)(t >> 8), micro = (int)(t & 255);
    const int ti = tile / tn, tj = tile - ti * tn;
    const int r = ((micro >> 6) << 2) | ((micro >> 2) & 3);
    const int c = (((micro >> 4) & 3) << 2) | (micro & 3);
    i = (ti << 4) | r;
    j = (tj << 4) | c;
}

}  // namespace ct
