// SELL view and value loaders shared by the sparse-product kernels.
#pragma once

#include "ct_internal.cuh"

namespace ct {

struct SellView {
    const int64_t* sp;   // slice offsets
    const int32_t* len;  // row lengths
    int64_t rows;
};

// Position of entry 0 of `row`; entry j sits at base + (j / 8) * 256 + j % 8.
__device__ __forceinline__ int64_t row_base(const SellView& m, int64_t row)
{
    return m.sp[row >> 5] + ((row & 31) << 3);
}
__device__ __forceinline__ int64_t chunk_pos(int64_t base, int64_t j) { return base + ((j >> 3) << 8) + (j & 7); }

template <typename VT>
struct Vals;

template <>
struct Vals<float> {
    static __device__ __forceinline__ void load8(const float* v, int64_t k, float (&o)[8])
    {
        const float4 a = __ldcs(reinterpret_cast<const float4*>(v + k));
        const float4 b = __ldcs(reinterpret_cast<const float4*>(v + k + 4));
        o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
        o[4] = b.x; o[5] = b.y; o[6] = b.z; o[7] = b.w;
    }
    static __device__ __forceinline__ float one(const float* v, int64_t k) { return __ldcs(v + k); }
};

template <>
struct Vals<__half> {
    static __device__ __forceinline__ void load8(const __half* v, int64_t k, float (&o)[8])
    {
        const uint4 a = __ldcs(reinterpret_cast<const uint4*>(v + k));
        const __half2* h = reinterpret_cast<const __half2*>(&a);
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const float2 f = __half22float2(h[t]);
            o[2 * t] = f.x;
            o[2 * t + 1] = f.y;
        }
    }
    static __device__ __forceinline__ float one(const __half* v, int64_t k)
    {
        return __half2float(__ldcs(v + k));
    }
};

}  // namespace ct
