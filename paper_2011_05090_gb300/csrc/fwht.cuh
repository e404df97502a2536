// Walsh-Hadamard transform of a 1024-row tile and the SRHT sample gather, shared by the
// fused update kernel and the sparse matrix-vector product.  (H_s = H_{s/1024} (x) H_1024,
// so output row a*1024 + b receives (-1)^popcount(a & t) (H_1024 z_t)[b] from tile t.)
#pragma once

#include "common.cuh"

namespace rgsdev {

constexpr int TILE = 1024;
constexpr int LOG_TILE = 10;
constexpr int TILE_THREADS = 256;    // 4 consecutive rows per thread

// Arithmetic of the transform for its value types (FP64, double-float pairs, or FP32).
template <typename V> struct FW;
template <> struct FW<double> {
    __device__ static double add(double a, double b) { return a + b; }
    __device__ static double sub(double a, double b) { return a - b; }
    __device__ static double neg(double a) { return -a; }
    __device__ static double shfl(double a, int m) { return __shfl_xor_sync(0xffffffffu, a, m); }
    __device__ static double from(double x) { return x; }
    __device__ static double from_float(float x) { return (double)x; }
    __device__ static double to_double(double a) { return a; }
    __device__ static double zero() { return 0.0; }
};
template <> struct FW<float> {        // the unique-precision setting: every butterfly in FP32
    __device__ static float add(float a, float b) { return a + b; }
    __device__ static float sub(float a, float b) { return a - b; }
    __device__ static float neg(float a) { return -a; }
    __device__ static float shfl(float a, int m) { return __shfl_xor_sync(0xffffffffu, a, m); }
    __device__ static float from(double x) { return __double2float_rn(x); }
    __device__ static float from_float(float x) { return x; }
    __device__ static double to_double(float a) { return (double)a; }
    __device__ static float zero() { return 0.f; }
};
template <> struct FW<df> {
    __device__ static df add(df a, df b) { return df_add(a, b); }
    __device__ static df sub(df a, df b) { return df_add(a, df_neg(b)); }
    __device__ static df neg(df a) { return df_neg(a); }
    __device__ static df shfl(df a, int m) {
        return {__shfl_xor_sync(0xffffffffu, a.h, m), __shfl_xor_sync(0xffffffffu, a.l, m)};
    }
    __device__ static df from(double x) {
        const float h = __double2float_rn(x);
        return {h, __double2float_rn(x - (double)h)};
    }
    __device__ static df from_float(float x) { return {x, 0.f}; }
    __device__ static double to_double(df a) { return (double)a.h + (double)a.l; }
    __device__ static df zero() { return {0.f, 0.f}; }
};

// Element b = 4*tid + e: bits 0-1 in registers, bits 2-6 across the warp, bits 7-9 through
// shared memory.  On return zt[b] holds (H_1024 z)[b] for every b.
template <typename V>
__device__ __forceinline__ void fwht_tile(V z[4], V* zt) {
    using F = FW<V>;
    V a0 = F::add(z[0], z[1]), a1 = F::sub(z[0], z[1]), a2 = F::add(z[2], z[3]), a3 = F::sub(z[2], z[3]);
    z[0] = F::add(a0, a2); z[1] = F::add(a1, a3); z[2] = F::sub(a0, a2); z[3] = F::sub(a1, a3);
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int s = 0; s < 5; ++s) {
        const int m = 1 << s;
        const bool upper = (lane & m) != 0;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const V o = F::shfl(z[e], m);
            z[e] = upper ? F::sub(o, z[e]) : F::add(z[e], o);
        }
    }
    __syncthreads();                               // previous readers of zt are done
#pragma unroll
    for (int e = 0; e < 4; ++e) zt[threadIdx.x * 4 + e] = z[e];
    __syncthreads();
    if (threadIdx.x < 128) {
        const int g = threadIdx.x;
        V v[8];
#pragma unroll
        for (int w = 0; w < 8; ++w) v[w] = zt[g + 128 * w];
#pragma unroll
        for (int h = 1; h < 8; h <<= 1)
#pragma unroll
            for (int a = 0; a < 8; a += 2 * h)
#pragma unroll
                for (int b = a; b < a + h; ++b) {
                    const V u = v[b], t = v[b + h];
                    v[b] = F::add(u, t);
                    v[b + h] = F::sub(u, t);
                }
#pragma unroll
        for (int w = 0; w < 8; ++w) zt[g + 128 * w] = v[w];
    }
    __syncthreads();
}

// Signs of D for the 4 rows r0..r0+3 (r0 a multiple of 4) applied to z, then the tile
// transform and the accumulation of every sampled output row into part[] (k entries).
template <typename V>
__device__ __forceinline__ void srht_tile(V z[4], int64_t r0, int64_t n, int tile, const uint32_t* signbits,
                                          const int32_t* srow, int k, V* zt, V* part) {
    using F = FW<V>;
    if (r0 < n) {
        const uint32_t bits = __ldg(signbits + (r0 >> 5)) >> (r0 & 31);
#pragma unroll
        for (int e = 0; e < 4; ++e)
            if ((bits >> e) & 1u) z[e] = F::neg(z[e]);
    }
    fwht_tile<V>(z, zt);
    for (int j = threadIdx.x; j < k; j += TILE_THREADS) {
        const int r = srow[j];
        const V v = zt[r & (TILE - 1)];
        part[j] = (__popc((r >> LOG_TILE) & tile) & 1) ? F::sub(part[j], v) : F::add(part[j], v);
    }
}

}  // namespace rgsdev
