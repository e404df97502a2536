// Sparse operator kernels of RGS-GMRES (Alg. 3 step 3, Sec. 4.2) and of the CGS2 comparator.
//  - spmv_sketch_kernel: w = A x for a tile of 1024 rows (CSR), stored, and its SRHT sketch
//    partials from the same registers (Alg. 2 step 1 for the next Arnoldi column).  With an
//    FP32/BF16 basis the products and sums run in double-float arithmetic on A's values
//    pre-split into float pairs (the paper allows a coarser matvec than u_fine as long as its
//    error stays O(u_crs), Sec. 4.1); with an FP64 basis everything is FP64.
//  - residual_kernel: r = b - A x in FP64 with per-CTA partial sums of r^2 (restart residual).
//  - sol_update_kernel: x += Q' cy (the GMRES solution update at the end of a cycle);
//    add_vector_kernel: x += z (a caller's preconditioner output, x = x0 + M (Q y)).
//  - hess_solve_kernel: y from the Givens-rotated Hessenberg system (one warp).
//  - multidot / axpy-style kernels for the CGS2 passes h = V^T w, w -= V h.
#include "fwht.cuh"

#include <algorithm>
#include <type_traits>
#include <vector>

using namespace rgsdev;

namespace {

__global__ void csr_split_df_kernel(const double* __restrict__ val, int64_t nnz, df* __restrict__ out) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
        const double v = val[e];
        const float h = __double2float_rn(v);
        out[e] = {h, __double2float_rn(v - (double)h)};
    }
}

// SELL-32 slice widths: the longest row of each slice of 32 rows (rows past n count as empty).
// The grid-stride loop runs over whole slices, so the 32 lanes of a warp share one slice.
__global__ void sell_width_kernel(int64_t n, const int32_t* __restrict__ rowptr, int64_t nslices,
                                  int32_t* __restrict__ width) {
    const int64_t rows = nslices * 32;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += (int64_t)gridDim.x * blockDim.x) {
        const int len = r < n ? rowptr[r + 1] - rowptr[r] : 0;
        const int wmax = (int)__reduce_max_sync(0xffffffffu, (unsigned)len);
        if ((r & 31) == 0) width[r >> 5] = wmax;
    }
}

// Fill the SELL-32 arrays: entry t of row r = 32 s + l goes to off[s] + 32 t + l; padding gets the
// value 0 and the column r (0 past n), a valid index.  col == nullptr: values only.
template <bool DFM>
__global__ void sell_fill_kernel(int64_t n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                                 const double* __restrict__ val, const int64_t* __restrict__ off, int64_t nslices,
                                 int32_t* __restrict__ col, void* __restrict__ out) {
    const int64_t rows = nslices * 32;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < rows; r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = r >> 5, q0 = off[s] + (r & 31);
        const int width = (int)((off[s + 1] - off[s]) >> 5);
        const int b0 = r < n ? rowptr[r] : 0, len = r < n ? rowptr[r + 1] - b0 : 0;
        for (int t = 0; t < width; ++t) {
            const int64_t q = q0 + 32 * (int64_t)t;
            const bool real = t < len;
            if (col) col[q] = real ? colind[b0 + t] : (r < n ? (int32_t)r : 0);
            const double v = real ? val[b0 + t] : 0.0;
            if constexpr (DFM) {
                const float h = __double2float_rn(v);
                reinterpret_cast<df*>(out)[q] = {h, __double2float_rn(v - (double)h)};
            } else {
                reinterpret_cast<double*>(out)[q] = v;
            }
        }
    }
}

template <typename TX> __device__ __forceinline__ float xf(const TX* x, int c) {
    if constexpr (sizeof(TX) == 2) return __bfloat162float(x[c]);
    else return (float)x[c];
}

// x[c] through the read-only path (x is not written by the kernel that reads it)
template <typename TX> __device__ __forceinline__ float xf_ro(const TX* x, int c) {
    if constexpr (sizeof(TX) == 2)
        return __bfloat162float(__ushort_as_bfloat16(__ldg(reinterpret_cast<const unsigned short*>(x) + c)));
    else return (float)__ldg(x + c);
}

// double-float product (ah + al) * b for an exact FP32 b (FMA gives the exact error of ah*b)
__device__ __forceinline__ df df_mul_f(df a, float b) {
    const float p = a.h * b;
    float e = fmaf(a.h, b, -p);
    e = fmaf(a.l, b, e);
    const float h = p + e;
    return {h, e - (h - p)};
}

struct SpmvParams {
    int64_t n;
    const int32_t* rowptr;
    const int32_t* colind;
    const double* val;      // FP64 values (FP64 mode)
    const df* vdf;          // double-float values (double-float mode)
    const void* x;
    const double* yscale;   // optional device scalar multiplying the FP64 product
    void* w;                // FP64 or double-float output
    const uint32_t* signbits;
    const int32_t* rows;
    int k;
    int ntiles;
    double* partials;
    const int* ctl;
    int64_t nslices;        // SELL-32 layout (the SELL kernels): slices, entry offsets, columns, values
    const int64_t* soff;
    const int32_t* scol;
    const void* sval;
};

// (A x) for the rows rbase + threadIdx.x + 256 e (e = 0..3) of a tile, stored to w and returned
// in z[e].  Lanes take consecutive rows, so a warp's row pointers, column indices, values and
// stores of w are contiguous.  PR rows at a time (one, in the launches below) go through three
// stages: the column indices and values of their first RB nonzeros, the gathers of x, the
// products (two accumulation chains per row).  Entries past the first RB of a row (none for
// the stencil operators of the workloads) are added one by one afterwards.
constexpr int RB = 8;

template <typename TX, bool DFM>
struct SpmvArith {
    using V = typename std::conditional<DFM, df, double>::type;
    using XV = typename std::conditional<DFM, float, double>::type;
    __device__ static XV xload(const TX* x, int c) {
        if constexpr (DFM) return xf(x, c);
        else return (double)x[c];
    }
    __device__ static XV xload_ro(const TX* x, int c) {       // x not written by the kernel
        if constexpr (DFM) return xf_ro(x, c);
        else return (double)__ldg(x + c);
    }
    __device__ static V vload(const SpmvParams& p, int q) {
        if constexpr (DFM) return p.vdf[q];
        else return __ldg(p.val + q);
    }
    __device__ static V madd(V acc, V v, XV xv) {
        if constexpr (DFM) return df_add(acc, df_mul_f(v, xv));
        else return fma(v, xv, acc);
    }
};

template <typename TX, bool DFM, int PR>
__device__ __forceinline__ void tile_rows(const SpmvParams& p, const TX* x, int64_t rbase,
                                          typename std::conditional<DFM, df, double>::type z[4]) {
    using AR = SpmvArith<TX, DFM>;
    using V = typename AR::V;
    using XV = typename AR::XV;
    int b0[4], b1[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int64_t r = rbase + threadIdx.x + (int64_t)TILE_THREADS * e;
        b0[e] = r < p.n ? __ldg(p.rowptr + r) : 0;
        b1[e] = r < p.n ? __ldg(p.rowptr + r + 1) : 0;
    }
#pragma unroll
    for (int e0 = 0; e0 < 4; e0 += PR) {
        int c[PR][RB];
        V v[PR][RB];
        XV xv[PR][RB];
#pragma unroll
        for (int h = 0; h < PR; ++h)
#pragma unroll
            for (int t = 0; t < RB; ++t) {
                const int q = b0[e0 + h] + t;
                if (q < b1[e0 + h]) {
                    c[h][t] = __ldg(p.colind + q);
                    v[h][t] = AR::vload(p, q);
                }
            }
#pragma unroll
        for (int h = 0; h < PR; ++h)
#pragma unroll
            for (int t = 0; t < RB; ++t)
                if (b0[e0 + h] + t < b1[e0 + h]) xv[h][t] = AR::xload(x, c[h][t]);
#pragma unroll
        for (int h = 0; h < PR; ++h) {
            const int e = e0 + h;
            V acc0 = FW<V>::zero(), acc1 = FW<V>::zero();
#pragma unroll
            for (int t = 0; t < RB; ++t)
                if (b0[e] + t < b1[e]) {
                    if (t & 1) acc1 = AR::madd(acc1, v[h][t], xv[h][t]);
                    else acc0 = AR::madd(acc0, v[h][t], xv[h][t]);
                }
            for (int q = b0[e] + RB; q < b1[e]; ++q) acc0 = AR::madd(acc0, AR::vload(p, q), AR::xload(x, __ldg(p.colind + q)));
            z[e] = FW<V>::add(acc0, acc1);
        }
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int64_t r = rbase + threadIdx.x + (int64_t)TILE_THREADS * e;
        if (r < p.n) {
            if constexpr (DFM) {
                reinterpret_cast<df*>(p.w)[r] = z[e];
            } else {
                if (p.yscale) z[e] *= *p.yscale;
                reinterpret_cast<double*>(p.w)[r] = z[e];
            }
        } else {
            z[e] = FW<V>::zero();
        }
    }
}

// tile_rows on the SELL-32 layout: warp w's 32 rows rbase + 256 e + 32 w + lane are one slice, so
// every load of entry t is one contiguous access and no row pointers are read.  Entries are
// multiplied and added exactly as in tile_rows (first RB alternately into two chains, the rest
// into the first); padding entries (value 0) add exact zeros, so the results are bit-identical.
// A, its SELL copy and x are read-only here (w is another buffer), so every load takes the
// read-only path and the four slices' offsets are read first and w is stored after the last
// product: no store orders a later slice's loads behind an earlier slice's, and the slices'
// load chains can overlap.
template <typename TX, bool DFM>
__device__ __forceinline__ void tile_rows_sell(const SpmvParams& p, const TX* x, int64_t rbase,
                                               typename std::conditional<DFM, df, double>::type z[4]) {
    using AR = SpmvArith<TX, DFM>;
    using V = typename AR::V;
    using XV = typename AR::XV;
    const int lane = threadIdx.x & 31;
    auto vld = [&](int64_t q) -> V {
        if constexpr (DFM) {
            const float2 t = __ldg(reinterpret_cast<const float2*>(p.sval) + q);
            return df{t.x, t.y};
        } else {
            return __ldg(reinterpret_cast<const double*>(p.sval) + q);
        }
    };
    int64_t q0[4];
    int width[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int64_t s = (rbase + (int64_t)TILE_THREADS * e + (threadIdx.x & ~31)) >> 5;   // warp-uniform
        q0[e] = 0;
        width[e] = 0;
        if (s < p.nslices) {
            q0[e] = __ldg(p.soff + s);
            width[e] = (int)((__ldg(p.soff + s + 1) - q0[e]) >> 5);
        }
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        V acc0 = FW<V>::zero(), acc1 = FW<V>::zero();
        int c[RB];
        V v[RB];
        XV xv[RB];
#pragma unroll
        for (int t = 0; t < RB; ++t)
            if (t < width[e]) {
                const int64_t q = q0[e] + 32 * t + lane;
                c[t] = __ldg(p.scol + q);
                v[t] = vld(q);
            }
#pragma unroll
        for (int t = 0; t < RB; ++t)
            if (t < width[e]) xv[t] = AR::xload_ro(x, c[t]);
#pragma unroll
        for (int t = 0; t < RB; ++t)
            if (t < width[e]) {
                if (t & 1) acc1 = AR::madd(acc1, v[t], xv[t]);
                else acc0 = AR::madd(acc0, v[t], xv[t]);
            }
        for (int t = RB; t < width[e]; ++t) {
            const int64_t q = q0[e] + 32 * t + lane;
            acc0 = AR::madd(acc0, vld(q), AR::xload_ro(x, __ldg(p.scol + q)));
        }
        z[e] = FW<V>::add(acc0, acc1);
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int64_t r = rbase + threadIdx.x + (int64_t)TILE_THREADS * e;
        if (r < p.n) {
            if constexpr (DFM) {
                reinterpret_cast<df*>(p.w)[r] = z[e];
            } else {
                if (p.yscale) z[e] *= *p.yscale;
                reinterpret_cast<double*>(p.w)[r] = z[e];
            }
        } else {
            z[e] = FW<V>::zero();
        }
    }
}

// FP64 values (DFM false) need more registers than 4 CTAs per SM leave (64): 3 CTAs, no spills.
template <typename TX, bool DFM, bool SRHT, bool SELL = false>
__global__ void __launch_bounds__(TILE_THREADS, DFM ? 4 : 3) spmv_sketch_kernel(SpmvParams p) {
    using V = typename std::conditional<DFM, df, double>::type;
    using F = FW<V>;
    extern __shared__ __align__(16) double smem[];
    V* zt = reinterpret_cast<V*>(smem);
    V* part = zt + TILE;
    int32_t* srow = reinterpret_cast<int32_t*>(part + (SRHT ? p.k : 0));
    pdl_wait();                        // the basis column and status of the kernel before
    pdl_launch_dependents();
    if (p.ctl != nullptr && (p.ctl[kStatusWord] != 0 || p.ctl[kStopWord] != 0)) return;
    const TX* x = reinterpret_cast<const TX*>(p.x);
    if (SRHT) {
        for (int j = threadIdx.x; j < p.k; j += TILE_THREADS) { srow[j] = p.rows[j]; part[j] = F::zero(); }
        __syncthreads();
    }
    for (int tile = blockIdx.x; tile < p.ntiles; tile += gridDim.x) {
        const int64_t rbase = (int64_t)tile * TILE;
        V z[4];
        if constexpr (SELL) tile_rows_sell<TX, DFM>(p, x, rbase, z);
        else tile_rows<TX, DFM, 1>(p, x, rbase, z);
        if (SRHT) {
            // the transform takes rows 4t .. 4t+3 in thread t: transpose through shared memory
            __syncthreads();                           // the previous tile's readers of zt are done
#pragma unroll
            for (int e = 0; e < 4; ++e) zt[threadIdx.x + TILE_THREADS * e] = z[e];
            __syncthreads();
#pragma unroll
            for (int e = 0; e < 4; ++e) z[e] = zt[threadIdx.x * 4 + e];
            srht_tile<V>(z, rbase + threadIdx.x * 4, p.n, tile, p.signbits, srow, p.k, zt, part);
        }
    }
    if (SRHT) {
        __syncthreads();
        V* out = reinterpret_cast<V*>(p.partials) + (int64_t)blockIdx.x * p.k;
        for (int j = threadIdx.x; j < p.k; j += TILE_THREADS) out[j] = part[j];
    }
}

// r = b - A x (FP64), per-CTA partial sums of r^2 in part[blockIdx.x]
__global__ void __launch_bounds__(256) residual_kernel(int64_t n, const int32_t* __restrict__ rowptr,
                                                       const int32_t* __restrict__ colind,
                                                       const double* __restrict__ val, const double* __restrict__ x,
                                                       const double* __restrict__ b, double* __restrict__ r,
                                                       double* __restrict__ part) {
    __shared__ double sh[8];
    double s2 = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double a = b[i];
        for (int q = rowptr[i]; q < rowptr[i + 1]; ++q) a = fma(-val[q], x[colind[q]], a);
        if (r) r[i] = a;
        s2 = fma(a, a, s2);
    }
    s2 = warp_sum(s2);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s2;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = threadIdx.x < 8 ? sh[threadIdx.x] : 0.0;
        t = warp_sum(t);
        if (threadIdx.x == 0) part[blockIdx.x] = t;
    }
}

// out[0] = sqrt(sum of part[0..np)) (one warp, fixed order)
__global__ void norm_final_kernel(const double* part, int np, double* out) {
    double v = 0.0;
    for (int b = threadIdx.x; b < np; b += 32) v += part[b];
    v = warp_sum(v);
    if (threadIdx.x == 0) out[0] = sqrt(v);
}

// sum of squares of a vector into per-CTA partials
__global__ void __launch_bounds__(256) sumsq_kernel(int64_t n, const double* __restrict__ v, double* __restrict__ part) {
    __shared__ double sh[8];
    double s2 = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        s2 = fma(v[i], v[i], s2);
    s2 = warp_sum(s2);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s2;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = threadIdx.x < 8 ? sh[threadIdx.x] : 0.0;
        t = warp_sum(t);
        if (threadIdx.x == 0) part[blockIdx.x] = t;
    }
}

// x += rowscale .* sum_{c < nsteps} Q'(:, c) cy[c]; nsteps from ctl[kStepsWord]
template <typename TQ>
__global__ void __launch_bounds__(256) sol_update_kernel(int64_t n, const TQ* __restrict__ Q, int64_t ldq,
                                                         const double* __restrict__ cy, double* __restrict__ x,
                                                         const int* ctl, const double* __restrict__ rowscale) {
    __shared__ df cdf[1024];
    __shared__ double cd[1024];
    const int nsteps = ctl[kStepsWord];
    if (ctl[kStatusWord] != 0 || nsteps <= 0) return;
    for (int c = threadIdx.x; c < nsteps && c < 1024; c += blockDim.x) {
        const double v = cy[c];
        const float h = __double2float_rn(v);
        cdf[c] = {h, __double2float_rn(v - (double)h)};
        cd[c] = v;
    }
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        if constexpr (sizeof(TQ) == 8) {
            double a = 0.0;
            for (int c = 0; c < nsteps; ++c) a = fma(Q[(int64_t)c * ldq + i], cd[c], a);
            x[i] += rowscale ? rowscale[i] * a : a;
        } else {
            df a = {0.f, 0.f};
            for (int c = 0; c < nsteps; ++c) {
                float q;
                if constexpr (sizeof(TQ) == 2) q = __bfloat162float(Q[(int64_t)c * ldq + i]);
                else q = Q[(int64_t)c * ldq + i];
                a = df_add(a, df_mul_f(cdf[c], q));
            }
            const double d = (double)a.h + (double)a.l;
            x[i] += rowscale ? rowscale[i] * d : d;
        }
    }
}

template <class TZ>
__global__ void __launch_bounds__(256) add_vector_kernel(int64_t n, const TZ* __restrict__ z, double* __restrict__ x,
                                                         const int* ctl) {
    if (ctl[kStatusWord] != 0) return;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] += (double)z[i];
}

// Back substitution on the rotated Hessenberg factor: Hr(0:j, 0:j) y = g(0:j), cy = sigma .* y.
// One warp; j = ctl[kStopWord] if the cycle stopped early, else jmax.  Writes ctl[kStepsWord] = j.
__global__ void hess_solve_kernel(const double* __restrict__ Hr, int ldh, const double* __restrict__ g,
                                  const double* __restrict__ colscale, int jmax, double* __restrict__ y,
                                  double* __restrict__ cy, int* ctl) {
    __shared__ double gs[1024];
    __shared__ double inv[1024];
    const int lane = threadIdx.x;
    if (ctl[kStatusWord] != 0) return;
    const int stop = ctl[kStopWord];
    const int j = stop > 0 ? stop : jmax;
    for (int t = lane; t < j; t += 32) {
        gs[t] = g[t];
        inv[t] = 1.0 / Hr[(size_t)t * ldh + t];
    }
    __syncwarp();
    for (int r = j - 1; r >= 0; --r) {
        const double yr = gs[r] * inv[r];
        for (int t = lane; t < r; t += 32) gs[t] = fma(-Hr[(size_t)r * ldh + t], yr, gs[t]);
        if (lane == 0) y[r] = yr;
        __syncwarp();
    }
    __syncwarp();
    for (int t = lane; t < j; t += 32) cy[t] = y[t] * (colscale ? colscale[t] : 1.0);
    if (lane == 0) ctl[kStepsWord] = j;
}

// CGS2 pass: partial dots part[blockIdx.x * ncols + c] = sum over the CTA's rows of V'(r, c) w(r).
// Warp w of the CTA handles columns c = w, w + 8, ...; lanes walk the CTA's row range.
__global__ void __launch_bounds__(256) multidot_kernel(int64_t n, const double* __restrict__ Vp, int64_t ldv,
                                                       int ncols, const double* __restrict__ w,
                                                       double* __restrict__ part, const int* ctl) {
    if (ctl[kStatusWord] != 0 || ctl[kStopWord] != 0) return;
    const int64_t per = (n + gridDim.x - 1) / gridDim.x;
    const int64_t r0 = (int64_t)blockIdx.x * per, r1 = min(n, r0 + per);
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    for (int c = wp; c < ncols; c += 8) {
        const double* v = Vp + (int64_t)c * ldv;
        double a0 = 0.0, a1 = 0.0;
        int64_t r = r0 + lane;
        for (; r + 32 < r1; r += 64) {
            a0 = fma(v[r], w[r], a0);
            a1 = fma(v[r + 32], w[r + 32], a1);
        }
        if (r < r1) a0 = fma(v[r], w[r], a0);
        const double t = warp_sum(a0 + a1);
        if (lane == 0) part[(int64_t)blockIdx.x * ncols + c] = t;
    }
}

// Sum the multidot partials over CTAs (warp per column): t[c]; coef[c] = sigma_c^2 t[c]; hacc[c] += t[c]
__global__ void multidot_reduce_kernel(const double* __restrict__ part, int np, int ncols,
                                       const double* __restrict__ sigma, double* __restrict__ coef,
                                       double* __restrict__ hacc, int accumulate, const int* ctl) {
    if (ctl[kStatusWord] != 0 || ctl[kStopWord] != 0) return;
    const int lane = threadIdx.x & 31;
    const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (c >= ncols) return;
    double v = 0.0;
    for (int b = lane; b < np; b += 32) v += part[(int64_t)b * ncols + c];
    v = warp_sum(v);
    if (lane == 0) {
        coef[c] = sigma[c] * sigma[c] * v;
        hacc[c] = accumulate ? hacc[c] + v : v;
    }
}

// w -= V' coef (FP64); optionally per-CTA partial sums of the updated w^2 and a copy into out
__global__ void __launch_bounds__(256) cgs_update_kernel(int64_t n, const double* __restrict__ Vp, int64_t ldv,
                                                         int ncols, const double* __restrict__ coef,
                                                         double* __restrict__ w, double* __restrict__ out,
                                                         double* __restrict__ part, const int* ctl) {
    __shared__ double sc[1024];
    __shared__ double sh[8];
    if (ctl[kStatusWord] != 0 || ctl[kStopWord] != 0) return;
    for (int c = threadIdx.x; c < ncols; c += blockDim.x) sc[c] = coef[c];
    __syncthreads();
    double s2 = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double a0 = w[i], a1 = 0.0;
        int c = 0;
        for (; c + 1 < ncols; c += 2) {
            a0 = fma(-Vp[(int64_t)c * ldv + i], sc[c], a0);
            a1 = fma(-Vp[(int64_t)(c + 1) * ldv + i], sc[c + 1], a1);
        }
        if (c < ncols) a0 = fma(-Vp[(int64_t)c * ldv + i], sc[c], a0);
        const double a = a0 + a1;
        w[i] = a;
        if (out) out[i] = a;
        s2 = fma(a, a, s2);
    }
    if (part) {
        s2 = warp_sum(s2);
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s2;
        __syncthreads();
        if (threadIdx.x < 32) {
            double t = threadIdx.x < 8 ? sh[threadIdx.x] : 0.0;
            t = warp_sum(t);
            if (threadIdx.x == 0) part[blockIdx.x] = t;
        }
    }
}

// dinv[r] = 1 / A(r, r) (0 flags a missing or zero diagonal in dinv_bad)
__global__ void jacobi_diag_kernel(int64_t n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                                   const double* __restrict__ val, double* __restrict__ dinv, int* bad) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        double d = 0.0;
        for (int q = rowptr[r]; q < rowptr[r + 1]; ++q)
            if (colind[q] == r) d += val[q];
        if (d == 0.0 || !isfinite(d)) { atomicExch(bad, 1); dinv[r] = 0.0; }
        else dinv[r] = 1.0 / d;
    }
}

// values of the column-scaled operator A D^{-1}
__global__ void jacobi_scale_kernel(int64_t nnz, const int32_t* __restrict__ colind, const double* __restrict__ val,
                                    const double* __restrict__ dinv, double* __restrict__ out) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x)
        out[e] = val[e] * dinv[colind[e]];
}

template <typename TX, bool DFM, bool SRHT, bool SELL = false>
void launch_spmv_t(rgs_context* ctx, const SpmvParams& p, int grid, size_t smem) {
    auto kern = spmv_sketch_kernel<TX, DFM, SRHT, SELL>;
    if (smem > 48 * 1024) RGS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    // programmatic serialization: scheduled while the kernel before is finishing (its CTAs wait
    // in pdl_wait for its completion)
    cudaLaunchAttribute attr{};
    attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr.val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(TILE_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = ctx->stream;
    cfg.attrs = &attr;
    cfg.numAttrs = ctx->pdl ? 1 : 0;
    RGS_CUDA(cudaLaunchKernelEx(&cfg, kern, p));
    ctx->launches++;
}

}  // namespace

void rgs_csr_split_df(rgs_context* ctx, const double* val, int64_t nnz, void* out) {
    const int grid = (int)std::min<int64_t>((nnz + 255) / 256, 4 * ctx->num_sms);
    csr_split_df_kernel<<<std::max(grid, 1), 256, 0, ctx->stream>>>(val, nnz, reinterpret_cast<df*>(out));
    RGS_CUDA(cudaGetLastError());
    ctx->launches++;
}

// One wave of resident CTAs: 4 per SM with double-float values (64 registers), 3 with FP64 values
// (80 registers: at 64 they spill).  Measured on the 128^3 RGMRES step (double-float):
// one row at a time at 4 CTAs per SM 178.0 us per step, at 3 CTAs per SM 184.7-185.5; two rows
// in flight at 2 CTAs per SM (128 registers) 193.1, two rows at 3 CTAs per SM (spilling) 197.6,
// four rows at 1 CTA per SM 226.8: occupancy hides the gathers better than rows in flight.
int rgs_spmv_nparts(const rgs_context* ctx, int64_t n, bool dfm) {
    const int ntiles = (int)((n + TILE - 1) / TILE);
    return std::max(1, std::min(ntiles, ctx->num_sms * (dfm ? 4 : 3)));   // one wave (launch bounds)
}

// w = A x (x in xtype; w FP64, or double-float when dfm), with SRHT partial sketches of w when sk != NULL.
int rgs_launch_spmv(rgs_context* ctx, const rgs_csr& A, const void* vdf, const void* x, int xtype, void* w, int dfm,
                    const rgs_sketch_obj* sk, double* partials, const int* ctl, const double* yscale,
                    const SellView* sell) {
    SpmvParams p{};
    RGS_REQUIRE(!(dfm && yscale), "scaled products are FP64 only");
    p.yscale = yscale;
    p.n = A.n;
    p.rowptr = A.rowptr;
    p.colind = A.colind;
    p.val = A.val;
    p.vdf = reinterpret_cast<const df*>(vdf);
    p.x = x;
    p.w = w;
    p.ctl = ctl;
    p.ntiles = (int)((A.n + TILE - 1) / TILE);
    const bool srht = sk != nullptr;
    if (srht) {
        p.signbits = sk->signbits.as<uint32_t>();
        p.rows = sk->rows.as<int32_t>();
        p.k = sk->k;
        p.partials = partials;
    }
    const int grid = rgs_spmv_nparts(ctx, A.n, dfm != 0);
    const size_t smem = srht ? TILE * 8 + (size_t)p.k * 8 + (size_t)((p.k + 3) & ~3) * 4 + 16 : 16;
    if (sell && srht) {
        RGS_REQUIRE(sell->nslices == (A.n + 31) / 32, "SELL layout of another operator");
        p.nslices = sell->nslices;
        p.soff = sell->off;
        p.scol = sell->col;
        p.sval = sell->val;
        if (dfm) {
            RGS_REQUIRE(xtype != RGS_F64, "double-float product needs an FP32 or BF16 vector");
            if (xtype == RGS_F32) launch_spmv_t<float, true, true, true>(ctx, p, grid, smem);
            else launch_spmv_t<__nv_bfloat16, true, true, true>(ctx, p, grid, smem);
        } else {
            if (xtype == RGS_F64) launch_spmv_t<double, false, true, true>(ctx, p, grid, smem);
            else if (xtype == RGS_F32) launch_spmv_t<float, false, true, true>(ctx, p, grid, smem);
            else launch_spmv_t<__nv_bfloat16, false, true, true>(ctx, p, grid, smem);
        }
        return grid;
    }
    if (dfm) {
        RGS_REQUIRE(xtype != RGS_F64, "double-float product needs an FP32 or BF16 vector");
        if (xtype == RGS_F32) {
            if (srht) launch_spmv_t<float, true, true>(ctx, p, grid, smem);
            else launch_spmv_t<float, true, false>(ctx, p, grid, smem);
        } else {
            if (srht) launch_spmv_t<__nv_bfloat16, true, true>(ctx, p, grid, smem);
            else launch_spmv_t<__nv_bfloat16, true, false>(ctx, p, grid, smem);
        }
    } else {
        if (xtype == RGS_F64) {
            if (srht) launch_spmv_t<double, false, true>(ctx, p, grid, smem);
            else launch_spmv_t<double, false, false>(ctx, p, grid, smem);
        } else if (xtype == RGS_F32) {
            if (srht) launch_spmv_t<float, false, true>(ctx, p, grid, smem);
            else launch_spmv_t<float, false, false>(ctx, p, grid, smem);
        } else {
            if (srht) launch_spmv_t<__nv_bfloat16, false, true>(ctx, p, grid, smem);
            else launch_spmv_t<__nv_bfloat16, false, false>(ctx, p, grid, smem);
        }
    }
    return grid;
}

bool rgs_build_sell(rgs_context* ctx, const rgs_csr& A, int dfm, SellBuf& sb) {
    const int64_t ns = (A.n + 31) / 32;
    if (ns == 0) return false;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((ns * 32 + 255) / 256, 4 * ctx->num_sms));
    DevBuf wd;
    wd.ensure(sizeof(int32_t) * (size_t)ns);
    sell_width_kernel<<<grid, 256, 0, ctx->stream>>>(A.n, A.rowptr, ns, wd.as<int32_t>());
    RGS_CUDA(cudaGetLastError());
    std::vector<int32_t> width((size_t)ns);
    RGS_CUDA(cudaMemcpyAsync(width.data(), wd.ptr, sizeof(int32_t) * (size_t)ns, cudaMemcpyDeviceToHost, ctx->stream));
    RGS_CUDA(cudaStreamSynchronize(ctx->stream));
    std::vector<int64_t> off((size_t)ns + 1);
    off[0] = 0;
    for (int64_t q = 0; q < ns; ++q) off[q + 1] = off[q] + 32 * (int64_t)width[q];
    if (off[ns] > A.nnz + A.nnz / 4) return false;
    sb.off.ensure(sizeof(int64_t) * (size_t)(ns + 1));
    RGS_CUDA(cudaMemcpyAsync(sb.off.ptr, off.data(), sizeof(int64_t) * (size_t)(ns + 1), cudaMemcpyHostToDevice,
                             ctx->stream));
    sb.col.ensure(sizeof(int32_t) * (size_t)std::max<int64_t>(off[ns], 1));
    sb.val.ensure(8 * (size_t)std::max<int64_t>(off[ns], 1));
    if (dfm)
        sell_fill_kernel<true><<<grid, 256, 0, ctx->stream>>>(A.n, A.rowptr, A.colind, A.val, sb.off.as<int64_t>(), ns,
                                                              sb.col.as<int32_t>(), sb.val.ptr);
    else
        sell_fill_kernel<false><<<grid, 256, 0, ctx->stream>>>(A.n, A.rowptr, A.colind, A.val, sb.off.as<int64_t>(), ns,
                                                               sb.col.as<int32_t>(), sb.val.ptr);
    RGS_CUDA(cudaGetLastError());
    RGS_CUDA(cudaStreamSynchronize(ctx->stream));          // the host offsets are read by the copy
    ctx->launches += 2;
    sb.nslices = ns;
    sb.entries = off[ns];
    return true;
}

void rgs_fill_sell_values(rgs_context* ctx, const rgs_csr& A, const double* val, int dfm, const SellBuf& sb,
                          DevBuf& out) {
    out.ensure(8 * (size_t)std::max<int64_t>(sb.entries, 1));
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((sb.nslices * 32 + 255) / 256, 4 * ctx->num_sms));
    if (dfm)
        sell_fill_kernel<true><<<grid, 256, 0, ctx->stream>>>(A.n, A.rowptr, A.colind, val, sb.off.as<int64_t>(),
                                                              sb.nslices, nullptr, out.ptr);
    else
        sell_fill_kernel<false><<<grid, 256, 0, ctx->stream>>>(A.n, A.rowptr, A.colind, val, sb.off.as<int64_t>(),
                                                               sb.nslices, nullptr, out.ptr);
    RGS_CUDA(cudaGetLastError());
    ctx->launches++;
}

int rgs_norm_grid(const rgs_context* ctx, int64_t n) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 2 * ctx->num_sms));
}

// r = b - A x; *norm_out (device) = ||r||
void rgs_launch_residual(rgs_context* ctx, const rgs_csr& A, const double* x, const double* b, double* r,
                         double* part, double* norm_out) {
    const int grid = rgs_norm_grid(ctx, A.n);
    residual_kernel<<<grid, 256, 0, ctx->stream>>>(A.n, A.rowptr, A.colind, A.val, x, b, r, part);
    RGS_CUDA(cudaGetLastError());
    norm_final_kernel<<<1, 32, 0, ctx->stream>>>(part, grid, norm_out);
    RGS_CUDA(cudaGetLastError());
    ctx->launches += 2;
}

void rgs_launch_norm(rgs_context* ctx, int64_t n, const double* v, double* part, double* norm_out) {
    const int grid = rgs_norm_grid(ctx, n);
    sumsq_kernel<<<grid, 256, 0, ctx->stream>>>(n, v, part);
    RGS_CUDA(cudaGetLastError());
    norm_final_kernel<<<1, 32, 0, ctx->stream>>>(part, grid, norm_out);
    RGS_CUDA(cudaGetLastError());
    ctx->launches += 2;
}

void rgs_launch_sol_update(rgs_context* ctx, int64_t n, const void* Q, int qtype, int64_t ldq, const double* cy,
                           double* x, const int* ctl, const double* rowscale) {
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 4 * ctx->num_sms));
    if (qtype == RGS_F64)
        sol_update_kernel<double><<<grid, 256, 0, ctx->stream>>>(n, (const double*)Q, ldq, cy, x, ctl, rowscale);
    else if (qtype == RGS_F32)
        sol_update_kernel<float><<<grid, 256, 0, ctx->stream>>>(n, (const float*)Q, ldq, cy, x, ctl, rowscale);
    else
        sol_update_kernel<__nv_bfloat16><<<grid, 256, 0, ctx->stream>>>(n, (const __nv_bfloat16*)Q, ldq, cy, x, ctl,
                                                                         rowscale);
    RGS_CUDA(cudaGetLastError());
    ctx->launches++;
}

void rgs_launch_add_vector(rgs_context* ctx, int64_t n, const void* z, int ztype, double* x, const int* ctl) {
    RGS_REQUIRE(ztype == RGS_F64 || ztype == RGS_F32, "z must be FP64 or FP32");
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 4 * ctx->num_sms));
    if (ztype == RGS_F64) add_vector_kernel<double><<<grid, 256, 0, ctx->stream>>>(n, (const double*)z, x, ctl);
    else add_vector_kernel<float><<<grid, 256, 0, ctx->stream>>>(n, (const float*)z, x, ctl);
    RGS_CUDA(cudaGetLastError());
    ctx->launches++;
}

void rgs_launch_hess_solve(rgs_context* ctx, const double* Hr, int ldh, const double* g, const double* colscale,
                           int jmax, double* y, double* cy, int* ctl) {
    hess_solve_kernel<<<1, 32, 0, ctx->stream>>>(Hr, ldh, g, colscale, jmax, y, cy, ctl);
    RGS_CUDA(cudaGetLastError());
    ctx->launches++;
}

int rgs_multidot_grid(const rgs_context* ctx, int64_t n) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + 1023) / 1024, 4 * ctx->num_sms));
}

void rgs_launch_cgs_pass(rgs_context* ctx, int64_t n, const double* Vp, int64_t ldv, int ncols, const double* sigma,
                         double* w, double* part, double* coef, double* hacc, int accumulate, const int* ctl) {
    const int grid = rgs_multidot_grid(ctx, n);
    multidot_kernel<<<grid, 256, 0, ctx->stream>>>(n, Vp, ldv, ncols, w, part, ctl);
    RGS_CUDA(cudaGetLastError());
    multidot_reduce_kernel<<<(ncols + 7) / 8, 256, 0, ctx->stream>>>(part, grid, ncols, sigma, coef, hacc,
                                                                       accumulate, ctl);
    RGS_CUDA(cudaGetLastError());
    ctx->launches += 2;
}

void rgs_launch_cgs_update(rgs_context* ctx, int64_t n, const double* Vp, int64_t ldv, int ncols, const double* coef,
                           double* w, double* out, double* part, const int* ctl) {
    const int grid = rgs_norm_grid(ctx, n);
    cgs_update_kernel<<<grid, 256, 0, ctx->stream>>>(n, Vp, ldv, ncols, coef, w, out, part, ctl);
    RGS_CUDA(cudaGetLastError());
    ctx->launches++;
}

// Right Jacobi preconditioning: dinv = diag(A)^{-1} and the values of A D^{-1}.
void rgs_launch_jacobi_setup(rgs_context* ctx, const rgs_csr& A, double* dinv, double* scaled_val) {
    int* bad = ctx->ctl.as<int>() + kFlagWord;
    RGS_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), ctx->stream));
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((A.n + 255) / 256, 4 * ctx->num_sms));
    jacobi_diag_kernel<<<grid, 256, 0, ctx->stream>>>(A.n, A.rowptr, A.colind, A.val, dinv, bad);
    RGS_CUDA(cudaGetLastError());
    jacobi_scale_kernel<<<grid, 256, 0, ctx->stream>>>(A.nnz, A.colind, A.val, dinv, scaled_val);
    RGS_CUDA(cudaGetLastError());
    int hbad = 0;
    RGS_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    RGS_CUDA(cudaStreamSynchronize(ctx->stream));
    RGS_REQUIRE(hbad == 0, "Jacobi preconditioner: zero or missing diagonal entry");
    ctx->launches += 2;
}
