// Alg. 2 steps 2, 5, 6 on the GPU: the sketched least-squares problem
// argmin_y ||S_{i-1} y - p_i|| solved through a Householder QR of S (the solver
// of the paper's experiments, Sec. 5), kept incrementally in compact-WY form
//     H_0 H_1 ... H_{i-1} = I - V T V^T,    S_i = (H_0 ... H_{i-1}) [R_S; 0],
// together with M = V T and R_S^{-1}.  With that form every phase is a parallel matrix-vector
// product spread over the whole GPU instead of i dependent reflector applications:
//   y  = [s, p] - V (M^T [s, p])         (apply the i existing reflectors: I - V T^T V^T)
//   new reflector H_i from y_s(i:k)      (appends s_i, column i of R_S = [y_s(0:i); beta])
//   x  = R_S^{-1} (H_i y_p)(0:i+1)       (the least-squares solution)
//   T(0:i, i) = -tau_i T V^T v_i, R_S^{-1} gains the column -R_S^{-1} y_s(0:i) / beta,
//   M(:, i) = V T(:, i) and N += v_i T(:, i)^T, N = V T^T (formed at the start of the next
//   launch; with N, T V^T v_i's sums over the rows below i are dots with N's columns, so the
//   new columns of T, R_S^{-1} and x are finished in the same phase as their other dots).
// One cooperative launch per column; its four phases are separated by three bounded grid
// barriers.
//
// Loads.  Vectors that every warp of the grid reads (T's new column, s', p, u, y, z) go through
// L1: a grid barrier ends with a GPU-scope acquire, after which ordinary loads see every write
// made before it, and none of these vectors is read, rewritten and read again within a launch.
// Through L2 alone (ld.cg) all 2432 warps fetch the same few lines from one L2 slice, which
// measured as most of each phase.  The per-CTA totals blk are the exception: rows written in
// one phase share lines with rows read in an earlier one, so they are read with ld.cg.
//
// Fine-precision arithmetic (u_fine).  GB300 runs FP64 at 2 operations per clock per SM, with
// about 65 cycles between dependent FP64 operations, against 128 FP32 operations per clock and
// about 5 cycles.  The kernel is therefore written once over an arithmetic type A:
//   FineF64  FP64 storage and arithmetic (FP64 bases, or on request);
//   FineDF   double-float storage and arithmetic (value hi + lo in two FP32 words, about 2^-48
//            relative error per operation), for FP32 / BF16 bases, where u_crs = 2^-24 or
//            2^-8: products by Dekker's TwoProduct through fmaf, sums by Knuth's TwoSum, dot
//            products accumulated as in Ogita, Rump and Oishi's Dot2 (a TwoSum chain of the
//            products' high parts plus one FP32 sum of all low-order terms).
// Squared norms (r_ii and ||p||) are summed in FP64 in both, for the exponent range, and every
// value leaving the kernel (R, x, sigma, S, ||p||) is FP64.
#include "common.cuh"
#include "givens.cuh"

#include <algorithm>
#include <type_traits>

using namespace rgsdev;

namespace {

constexpr int LT = 512;        // threads per CTA (one CTA per SM)
constexpr int NW = LT / 32;    // warps per CTA
constexpr int kTotMax = 8;     // per-CTA totals are read for up to 32 * kTotMax CTAs at once

// ------------------------------------------------------------------ arithmetic types
struct FineF64 {
    using T = double;
    struct Acc {
        double v;
    };
    __device__ static T zero() { return 0.0; }
    __device__ static T one() { return 1.0; }
    __device__ static T from_d(double x) { return x; }
    __device__ static double to_d(T x) { return x; }
    __device__ static T add(T a, T b) { return a + b; }
    __device__ static T sub(T a, T b) { return a - b; }
    __device__ static T mul(T a, T b) { return a * b; }
    __device__ static T neg(T a) { return -a; }
    __device__ static T div(T a, T b) { return a / b; }
    __device__ static T sqrt_(T a) { return sqrt(a); }
    __device__ static bool is_zero(T a) { return a == 0.0; }
    __device__ static bool nonneg(T a) { return a >= 0.0; }
    __device__ static T wsum(T v) { return warp_sum(v); }
    __device__ static T shfl_xor(T v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
    __device__ static T ld(const double* p) { return *p; }
    __device__ static T ldcg(const double* p) { return __ldcg(p); }
    __device__ static void st(double* p, T v) { *p = v; }
    __device__ static Acc acc0() { return {0.0}; }
    __device__ static void acc(Acc& s, T a, T b) { s.v = fma(a, b, s.v); }
    __device__ static T val(Acc s) { return s.v; }
    __device__ static double round_d(double x) { return x; }            // a scalar as this arithmetic keeps it
    __device__ static double recip_d(double y) { return 1.0 / y; }
};

__device__ __forceinline__ df df_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bv = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bv)), __fsub_rn(b, bv))};
}
__device__ __forceinline__ df df_fast(float a, float b) {      // |a| >= |b| or a = 0
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

struct FineDF {
    using T = df;
    struct Acc {
        float s, c;           // running sum of the products' high parts, FP32 sum of the rest
    };
    __device__ static T zero() { return {0.f, 0.f}; }
    __device__ static T one() { return {1.f, 0.f}; }
    __device__ static T from_d(double x) {
        const float h = __double2float_rn(x);
        return {h, __double2float_rn(x - (double)h)};
    }
    __device__ static double to_d(T x) { return (double)x.h + (double)x.l; }
    __device__ static T add(T a, T b) {
        const df s = df_two_sum(a.h, b.h);
        return df_fast(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
    }
    __device__ static T neg(T a) { return {-a.h, -a.l}; }
    __device__ static T sub(T a, T b) { return add(a, neg(b)); }
    __device__ static T mul(T a, T b) {
        const float p = __fmul_rn(a.h, b.h);
        float e = __fmaf_rn(a.h, b.h, -p);
        e = __fmaf_rn(a.h, b.l, e);
        e = __fmaf_rn(a.l, b.h, e);
        return df_fast(p, e);
    }
    // a / b: quotient of the high words, corrected once by the remainder a - q b
    __device__ static T div(T a, T b) {
        const float q1 = __fdiv_rn(a.h, b.h);
        const T r = sub(a, mul(b, {q1, 0.f}));
        const float q2 = __fdiv_rn(r.h, b.h);
        return df_fast(q1, q2);
    }
    // sqrt(a): FP32 root of the high word and one Newton correction in double-float
    __device__ static T sqrt_(T a) {
        if (!(a.h > 0.f)) return {sqrtf(a.h), 0.f};
        const float y = sqrtf(a.h);
        const float p = __fmul_rn(y, y);
        const float e = __fmaf_rn(y, y, -p);
        const float d = __fadd_rn(__fsub_rn(__fsub_rn(a.h, p), e), a.l);
        return df_fast(y, __fdiv_rn(d, __fmul_rn(2.f, y)));
    }
    __device__ static bool is_zero(T a) { return a.h == 0.f && a.l == 0.f; }
    __device__ static bool nonneg(T a) { return a.h > 0.f || (a.h == 0.f && a.l >= 0.f); }
    __device__ static T wsum(T v) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const T t = {__shfl_xor_sync(0xffffffffu, v.h, o), __shfl_xor_sync(0xffffffffu, v.l, o)};
            v = add(v, t);    // TwoSum is exact, so both lanes of a pair get the same bits
        }
        return v;
    }
    __device__ static T shfl_xor(T v, int o) {
        return {__shfl_xor_sync(0xffffffffu, v.h, o), __shfl_xor_sync(0xffffffffu, v.l, o)};
    }
    __device__ static T ld(const double* p) {
        const float2 v = *reinterpret_cast<const float2*>(p);
        return {v.x, v.y};
    }
    __device__ static T ldcg(const double* p) {
        const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
        return {v.x, v.y};
    }
    __device__ static void st(double* p, T v) { *reinterpret_cast<float2*>(p) = make_float2(v.h, v.l); }
    __device__ static Acc acc0() { return {0.f, 0.f}; }
    __device__ static void acc(Acc& s, T a, T b) {
        const float p = __fmul_rn(a.h, b.h);
        float e = __fmaf_rn(a.h, b.h, -p);
        e = __fmaf_rn(a.h, b.l, e);
        e = __fmaf_rn(a.l, b.h, e);
        const df t = df_two_sum(s.s, p);
        s.s = t.h;
        s.c = __fadd_rn(s.c, __fadd_rn(t.l, e));
    }
    __device__ static T val(Acc s) { return df_fast(s.s, s.c); }
    __device__ static double round_d(double x) { return x; }
    __device__ static double recip_d(double y) { return 1.0 / y; }
};

// FP32 storage and arithmetic: the unique-precision setting of Sec. 5.1 (u_fine = u_crs = FP32).
// Values live in the first four bytes of the 8-byte slots; the squared norms are FP32 sums too,
// and r_ii, its reciprocal and ||p|| are FP32 numbers.
struct FineF32 {
    using T = float;
    struct Acc {
        float v;
    };
    __device__ static T zero() { return 0.f; }
    __device__ static T one() { return 1.f; }
    __device__ static T from_d(double x) { return __double2float_rn(x); }
    __device__ static double to_d(T x) { return (double)x; }
    __device__ static T add(T a, T b) { return __fadd_rn(a, b); }
    __device__ static T sub(T a, T b) { return __fsub_rn(a, b); }
    __device__ static T mul(T a, T b) { return __fmul_rn(a, b); }
    __device__ static T neg(T a) { return -a; }
    __device__ static T div(T a, T b) { return __fdiv_rn(a, b); }
    __device__ static T sqrt_(T a) { return sqrtf(a); }
    __device__ static bool is_zero(T a) { return a == 0.f; }
    __device__ static bool nonneg(T a) { return a >= 0.f; }
    __device__ static T wsum(T v) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = __fadd_rn(v, __shfl_xor_sync(0xffffffffu, v, o));
        return v;
    }
    __device__ static T shfl_xor(T v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
    __device__ static T ld(const double* p) { return *reinterpret_cast<const float*>(p); }
    __device__ static T ldcg(const double* p) { return __ldcg(reinterpret_cast<const float*>(p)); }
    __device__ static void st(double* p, T v) { *reinterpret_cast<float*>(p) = v; }
    __device__ static Acc acc0() { return {0.f}; }
    __device__ static void acc(Acc& s, T a, T b) { s.v = __fmaf_rn(a, b, s.v); }
    __device__ static T val(Acc s) { return s.v; }
    __device__ static double round_d(double x) { return (double)__double2float_rn(x); }
    __device__ static double recip_d(double y) { return (double)__fdiv_rn(1.f, __double2float_rn(y)); }
};

// ------------------------------------------------------------------ reductions
// Block-wide sums of N values held by lane 0 of each warp (other lanes ignored): one warp
// adds the NW per-warp values.  Identical in every thread; sm holds >= N * (NW + 1) values.
template <class A, int N>
__device__ __forceinline__ void block_sum_lane0(typename A::T (&v)[N], typename A::T* sm) {
    using T = typename A::T;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < N; ++q) sm[q * NW + w] = v[q];
    __syncthreads();
    if (threadIdx.x < 32) {
#pragma unroll
        for (int q = 0; q < N; ++q) {
            T t = lane < NW ? sm[q * NW + lane] : A::zero();
            t = A::wsum(t);
            if (lane == 0) sm[N * NW + q] = t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < N; ++q) v[q] = sm[N * NW + q];
}

// Deterministic totals of the per-CTA values blk[b*4 + off], blk[b*4 + off + 1] (type A::T),
// computed by one whole warp (all its loads issued at once) and valid in all its lanes.
template <class A>
__device__ void warp_total2(const double* blk, int off, typename A::T& t0, typename A::T& t1) {
    using T = typename A::T;
    const int lane = threadIdx.x & 31, G = gridDim.x;
    T a0[kTotMax], a1[kTotMax];
#pragma unroll
    for (int q = 0; q < kTotMax; ++q) {
        const int b = lane + 32 * q;
        a0[q] = b < G ? A::ldcg(blk + (size_t)b * 4 + off) : A::zero();
        a1[q] = b < G ? A::ldcg(blk + (size_t)b * 4 + off + 1) : A::zero();
    }
    T v0 = A::zero(), v1 = A::zero();
#pragma unroll
    for (int q = 0; q < kTotMax; ++q)
        if (32 * q < G) { v0 = A::add(v0, a0[q]); v1 = A::add(v1, a1[q]); }
    t0 = A::wsum(v0);
    t1 = A::wsum(v1);
}

// Sum over b = b0, b0 + step, ... < b1 of the partial sketch entries src[b * k + l] (double-float
// or FP64), written by an earlier launch, in the arithmetic of A.
template <class A>
__device__ __forceinline__ typename A::T part_sum(const double* src, bool sdf, int b0, int b1, int step, int k,
                                                  int l) {
    if constexpr (std::is_same<typename A::T, float>::value) {
        // unique precision: the FP32 partials (high words of the pairs) summed in FP32
        const df* d = reinterpret_cast<const df*>(src);
        float t0 = 0.f, t1 = 0.f;
        for (int bb = b0; bb < b1; bb += 16 * step) {
            float v[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int b = bb + q * step;
                v[q] = b < b1 ? (sdf ? d[(size_t)b * k + l].h : __double2float_rn(src[(size_t)b * k + l])) : 0.f;
            }
#pragma unroll
            for (int q = 0; q < 16; q += 2) {
                t0 = __fadd_rn(t0, v[q]);
                t1 = __fadd_rn(t1, v[q + 1]);
            }
        }
        return __fadd_rn(t0, t1);
    }
    if (sdf) {
        const df* d = reinterpret_cast<const df*>(src);
        df t0 = {0.f, 0.f}, t1 = {0.f, 0.f};
        for (int bb = b0; bb < b1; bb += 16 * step) {  // 16 loads in flight, then the sums
            df v[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int b = bb + q * step;
                v[q] = b < b1 ? d[(size_t)b * k + l] : df{0.f, 0.f};
            }
#pragma unroll
            for (int q = 0; q < 16; q += 2) {
                t0 = df_add(t0, v[q]);
                t1 = df_add(t1, v[q + 1]);
            }
        }
        t0 = df_add(t0, t1);
        if constexpr (std::is_same<typename A::T, df>::value)
            return t0;
        else
            return (double)t0.h + (double)t0.l;
    }
    double v0 = 0.0, v1 = 0.0, v2 = 0.0, v3 = 0.0;
    int b = b0;
#pragma unroll 2
    for (; b + 3 * step < b1; b += 4 * step) {
        v0 += src[(size_t)b * k + l];
        v1 += src[(size_t)(b + step) * k + l];
        v2 += src[(size_t)(b + 2 * step) * k + l];
        v3 += src[(size_t)(b + 3 * step) * k + l];
    }
    for (; b < b1; b += step) v0 += src[(size_t)b * k + l];
    return A::from_d((v0 + v1) + (v2 + v3));
}

// Dot products of a row (stride 1, entries [0, jend)) with vectors y1 and y2, a warp with lanes
// over the entries: the lane partials summed over the warp, valid in every lane; use1 / use2
// select the vectors needed.
template <class A>
__device__ __forceinline__ void warp_row_dot2(const double* row, const double* y1, const double* y2, int jend,
                                              bool use1, bool use2, typename A::T& o1, typename A::T& o2) {
    const int lane = threadIdx.x & 31;
    typename A::Acc a1[4] = {A::acc0(), A::acc0(), A::acc0(), A::acc0()};
    typename A::Acc a2[4] = {A::acc0(), A::acc0(), A::acc0(), A::acc0()};
    // blocks of 4 x 32 entries: every load of a block is issued before its arithmetic
    for (int j0 = 0; j0 < jend; j0 += 128) {
        typename A::T v[4], w1[4], w2[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int j = j0 + 32 * q + lane;
            const bool ok = j < jend;
            v[q] = ok ? A::ld(row + j) : A::zero();
            w1[q] = (ok && use1) ? A::ld(y1 + j) : A::zero();
            w2[q] = (ok && use2) ? A::ld(y2 + j) : A::zero();
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (use1) A::acc(a1[q], v[q], w1[q]);
            if (use2) A::acc(a2[q], v[q], w2[q]);
        }
    }
    o1 = use1 ? A::wsum(A::add(A::add(A::val(a1[0]), A::val(a1[1])), A::add(A::val(a1[2]), A::val(a1[3]))))
              : A::zero();
    o2 = use2 ? A::wsum(A::add(A::add(A::val(a2[0]), A::val(a2[1])), A::add(A::val(a2[2]), A::val(a2[3]))))
              : A::zero();
}

// Step 2 by the normal equations S^T S x = S^T p with two Richardson sweeps from x = 0 (the
// alternative Sec. 2.3 names for larger S): x1 = S^T p, x2 = x1 + S^T (p - S x1), FP64.  Entered
// after phase 1 with r_ii known; S(:, i) = s'_i / r_ii is appended here, with a row-major copy in
// the V^T slot (unused in this mode) for the row products.  Three grid phases:
//   1b: S(:, i) and its row copy; x1_j = S(:, j) . p for j < i and x1_i = (s' . p) / r_ii (warp per j)
//   2:  r_l = p_l - S(l, 0:i+1) x1 (warp per row)
//   3:  x2_j = x1_j + S(:, j) . r (warp per j), written to R(:, xcol) and the step-3 coefficients.
__device__ __forceinline__ void richardson_phases(const LSState& st, const LSStep& a, GridBarrier& bar, int* ctl,
                                               double inv_r, double pmul, unsigned long long* tr) {
    const int k = st.k, mm = st.mmax, i = a.i;
    const int G = gridDim.x, tid = threadIdx.x, lane = tid & 31;
    const int nthreads = G * LT, gtid = blockIdx.x * LT + tid;
    const int gwarp = blockIdx.x + G * (tid >> 5), nwarps = nthreads >> 5;
    const bool app = a.append != 0, sol = a.solve != 0;
    auto coldot = [&](const double* u, const double* v) {     // sum_l u_l v_l over k rows, a warp
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
        int l = lane;
        for (; l + 96 < k; l += 128) {
            s0 = fma(u[l], v[l], s0);
            s1 = fma(u[l + 32], v[l + 32], s1);
            s2 = fma(u[l + 64], v[l + 64], s2);
            s3 = fma(u[l + 96], v[l + 96], s3);
        }
        for (; l < k; l += 32) s0 = fma(u[l], v[l], s0);
        return warp_sum((s0 + s1) + (s2 + s3));
    };
    if (app)
        for (int l = gtid; l < k; l += nthreads) {
            const double sl = st.sbuf[l] * inv_r;
            st.S[(size_t)i * k + l] = sl;
            st.VT[(size_t)l * mm + i] = sl;
        }
    if (sol)
        for (int j = gwarp; j <= i; j += nwarps) {
            const double d = j < i ? coldot(st.S + (size_t)j * k, st.pbuf) : coldot(st.sbuf, st.pbuf) * inv_r;
            if (lane == 0) st.u2p[j] = d * pmul;
        }
    if (!bar.sync(ctl, tr ? tr + 3 : nullptr)) return;
    if (!sol) {
        if (tr) tr[9] = globaltimer();
        return;
    }
    for (int l = gwarp; l < k; l += nwarps) {
        const double* row = st.VT + (size_t)l * mm;
        double s0 = 0.0, s1 = 0.0;
        int j = lane;
        for (; j + 32 <= i; j += 64) {
            s0 = fma(row[j], st.u2p[j], s0);
            s1 = fma(row[j + 32], st.u2p[j + 32], s1);
        }
        if (j <= i) s0 = fma(row[j], st.u2p[j], s0);
        const double d = warp_sum(s0 + s1);
        if (lane == 0) st.yp[l] = st.pbuf[l] * pmul - d;
    }
    if (!bar.sync(ctl, tr ? tr + 5 : nullptr)) return;
    for (int j = gwarp; j <= i; j += nwarps) {
        const double d = coldot(st.S + (size_t)j * k, st.yp);
        if (lane == 0) {
            const double x = st.u2p[j] + d;
            st.R[(size_t)a.xcol * st.ldr + j] = x;
            st.coef[j] = x * st.sigma[j];
        }
    }
    if (tr) tr[9] = globaltimer();
}

// GMRES (one warp): rotates H(:, i-1) = [R(0:i, i); r_ii] by the stored rotations, forms the next
// one and updates g; sets the stop word when the least-squares residual reaches the tolerance
// or the launch found a breakdown.
__device__ __forceinline__ void givens_and_stop(const LSState& st, const LSStep& a, double r, int* ctl,
                                                bool breakdown) {
    const int i = a.i;
    const double* rc = st.R + (size_t)i * st.ldr;
    auto hcol = [&](int t) { return t < i ? rc[t] : r; };
    const double res = givens_column_warp<true>(i - 1, hcol, st.cs, st.sn, st.g, st.Hr, st.mmax);
    if (threadIdx.x == 0 && (breakdown || res <= a.stop_tol)) atomicCAS(ctl + kStopWord, 0, i);
}

template <class A>
__global__ void __launch_bounds__(LT, 1) ls_kernel(LSState st, LSStep a) {
    using T = typename A::T;
    using Acc = typename A::Acc;
    __shared__ T shT[2 * (NW + 1) + 2];        // A::T block sums and totals
    __shared__ T qs[3 * NW];                   // per-warp partial dots of the column phases
    __shared__ T shP[NW * 32];                 // phase 0: the warps' range sums of one segment
    __shared__ T scT[8];                       // scalars of the current phase, in A::T
    __shared__ double sc[8];                   // FP64 scalars of phase 1
    int* ctl = st.ctl;
    pdl_wait();                        // the partial sketches and status of the kernel before
    pdl_launch_dependents();
    if (ctl[kStatusWord] != 0 || ctl[kStopWord] != 0) return;
    const int k = st.k, mm = st.mmax, i = a.i;
    const int G = gridDim.x;
    const int tid = threadIdx.x, lane = tid & 31;
    const int nthreads = G * LT, gtid = blockIdx.x * LT + tid;
    // warp w of CTA b is global warp b + G*w, so consecutive items spread over all SMs
    const int gwarp = blockIdx.x + G * (tid >> 5), nwarps = nthreads >> 5;
    const bool app = a.append != 0, sol = a.solve != 0;
    const bool p_parts = sol && a.p_vec == nullptr;
    constexpr bool f64 = std::is_same<A, FineF64>::value;
    const bool rich = f64 && a.rich != 0;               // Richardson sweeps instead of the reflectors
    const T zero = A::zero();
    // optional timestamps, thread 0 of every CTA: start, then arrival at and departure from each
    // grid barrier (slots 1, 2 for the first, 3, 4 for the second, ...), end in slot 9
    unsigned long long* tr = (a.trace != nullptr && tid == 0) ? a.trace + (size_t)blockIdx.x * kLsTraceSlots : nullptr;
    if (tr) tr[0] = globaltimer();
    GridBarrier bar(ctl);
    const double pref = (app && tid == 0) ? st.pnorm[i] : 0.0;   // ||p_i||, for the breakdown test
    const int nfold0 = *st.nfold;                                // reflectors in N before this launch
    // N must hold reflectors 0 .. i-2 (or already i-1: a retried step); anything else (a launch
    // that gave up between phase 0 and its first barrier) leaves it unusable: every CTA reads the
    // same word and leaves before any write
    if (app && !rich && i > 0 && nfold0 != i - 1 && nfold0 != i) {
        if (gtid == 0 && ctl[kStatusWord] == 0 && ctl[kStopWord] == 0) {
            atomicCAS(ctl + kStatusWord, 0, (int)RGS_ERR_INVALID_ARG);
            ctl[kDetailWord] = i;
        }
        return;
    }
    if (tid == 0) {                                              // the partial sketches' scales
        scT[6] = A::from_d(a.s_scale);
        scT[7] = A::from_d(a.p_scale);
    }

    __syncthreads();
    const T s_scale = scT[6], p_scale = scT[7];

    // ---- phase 0: the totals of s' and p.  Item = (segment of R rows, vector), R the largest of
    //      32, 16, 8, 4 that still gives at least G/2 items (small k: shorter segments spread the
    //      sums over more CTAs; one item per CTA, as each item has a fixed serial part).  The
    //      item's NW warps sum consecutive ranges of the partial sketches;
    //      within a warp, lane = (row, slice): slice t of the 32/R takes every (32/R)-th partial
    //      of the range and the slices are combined by shuffles.  Warp 0 adds the NW range sums
    //      in a fixed pairwise order (deterministic), scales and stores them and forms the squared norms (FP64).
    //      Then every warp forms rows of M(:, i-1) = V(:, 0:i) T(0:i, i-1).
    {
        const int warp = tid >> 5;
        constexpr bool f32 = std::is_same<T, float>::value;   // unique precision: FP32 squared norms
        double nrm_s = 0.0, nrm_p = 0.0;               // warp 0, lane 0
        float nrm_sf = 0.f, nrm_pf = 0.f;
        int R = 32;
        while (R > 4 && 2 * 2 * ((k + R - 1) / R) < G) R >>= 1;
        const int S = 32 / R, rl = lane & (R - 1), sl = lane / R;
        const int nseg = (k + R - 1) / R;
        const int nitems = nseg * 2;
        for (int it = blockIdx.x; it < nitems; it += G) {
            const int seg = it >> 1, vec = it & 1;       // vec 0: s', vec 1: p (uniform over the CTA)
            if (vec == 0 ? !app : !sol) continue;
            const int l = seg * R + rl;
            T part = zero;
            if (vec == 0 || p_parts) {
                const int np = vec == 0 ? a.s_nparts : a.p_nparts;
                const int chunk = (np + NW - 1) / NW;
                const int b0 = min(np, warp * chunk), b1 = min(np, b0 + chunk);
                if (l < k && b0 + sl < b1)
                    part = part_sum<A>(vec == 0 ? a.s_part : a.p_part, (vec == 0 ? a.s_df : a.p_df) != 0, b0 + sl, b1,
                                       S, k, l);
                for (int o = R; o < 32; o <<= 1) part = A::add(part, A::shfl_xor(part, o));
            } else if (warp == 0 && l < k) {
                part = A::from_d(a.p_vec[l]);
            }
            if (tr && it == (int)blockIdx.x) tr[11] = globaltimer();   // this thread's sums
            if (sl == 0) shP[warp * 32 + rl] = part;
            __syncthreads();
            if (tr && it == (int)blockIdx.x) tr[12] = globaltimer();
            if (warp == 0) {
                const int lw = seg * R + lane;           // lanes 0..R-1: the segment's rows
                const bool own = lane < R && lw < k;
                T t[NW];                                 // the NW range sums, added as a pairwise tree
#pragma unroll
                for (int w = 0; w < NW; ++w) t[w] = lane < R ? shP[w * 32 + lane] : zero;
#pragma unroll
                for (int h = 1; h < NW; h *= 2)
#pragma unroll
                    for (int w = 0; w + h < NW; w += 2 * h) t[w] = A::add(t[w], t[w + h]);
                T v = t[0];
                v = A::mul(v, vec == 0 ? s_scale : p_scale);
                double vd = 0.0;
                if (own) {
                    A::st((vec == 0 ? st.sbuf : st.pbuf) + lw, v);
                    vd = A::to_d(v);
                    if (vec == 1 && a.p_store) a.p_store[lw] = vd;
                }
                if constexpr (f32) {
                    const float vf = own ? (float)vd : 0.f;
                    const float sq = A::wsum(__fmul_rn(vf, vf));
                    if (vec == 0) nrm_sf = __fadd_rn(nrm_sf, sq); else nrm_pf = __fadd_rn(nrm_pf, sq);
                } else {
                    const double sq = warp_sum(vd * vd);
                    if (vec == 0) nrm_s += sq; else nrm_p += sq;
                }
            }
            if (tr && it == (int)blockIdx.x) tr[13] = globaltimer();
            __syncthreads();                               // shP is reused by the next item
        }
        if (tr) tr[10] = globaltimer();
        if (i > 0 && !rich) {
            // M(:, i-1) = V(:, 0:i) T(0:i, i-1): T's column i-1 was completed by the previous
            // launch; warp per row of the row-major copy VT, lanes over the columns
            const double* tc = st.T + (size_t)(i - 1) * mm;
            for (int l = gwarp; l < k; l += nwarps) {
                T d, unused;
                warp_row_dot2<A>(st.VT + (size_t)l * mm, tc, tc, min(i, l + 1), true, false, d, unused);
                if (lane == 0) A::st(st.M + (size_t)(i - 1) * k + l, d);
            }
            // N = V T^T (column-major k x mmax) gains reflector i - 1: N(:, j) += V(:, i-1) T(j, i-1)
            // for j < i - 1, N(:, i-1) = V(:, i-1) T(i-1, i-1); V(:, i-1) vanishes above row i - 1.
            // Once per reflector: nfold counts the reflectors in N (a step that is solved and then
            // appended, or retried after a failed launch, reaches this with the same i again).
            if (app && nfold0 == i - 1) {
                const int r0 = (i - 1) & ~15;                 // item rows from a 16-row boundary
                const int nch = (k - r0 + 255) / 256;
                const double* vc = st.V + (size_t)(i - 1) * k;
                for (int item = gwarp; item < i * nch; item += nwarps) {   // (column, 256 rows)
                    const int j = item / nch, l0 = r0 + 256 * (item % nch);
                    const T tj = A::ld(tc + j);
                    double* nc = st.N + (size_t)j * k;
                    T nv[8], vv[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const int l = l0 + 32 * q + lane;
                        vv[q] = l < k ? A::ld(vc + l) : zero;
                        nv[q] = (l < k && j < i - 1) ? A::ld(nc + l) : zero;
                    }
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const int l = l0 + 32 * q + lane;
                        if (l < k) A::st(nc + l, A::add(nv[q], A::mul(vv[q], tj)));
                    }
                }
            }
        }
        if (tid == 0) {
            if constexpr (f32) {
                A::st(st.blk + blockIdx.x * 4 + 0, nrm_sf);
                A::st(st.blk + blockIdx.x * 4 + 1, nrm_pf);
            } else {
                st.blk[blockIdx.x * 4 + 0] = nrm_s;
                st.blk[blockIdx.x * 4 + 1] = nrm_p;
            }
        }
    }
    if (!bar.sync(ctl, tr ? tr + 1 : nullptr)) return;
    if (app && !rich && gtid == 0) *st.nfold = i;

    // ---- phase 1: r_ii, s_i = s'/r_ii; u2 = M(:, 0:i)^T [s, p] = T^T V^T [s, p]
    // Warp 0 reads the squared norms' totals and forms the phase's scalars (FP64 square roots
    // and divisions are long sequences on the FP64 pipe, so no other warp repeats them) while
    // warps 4..15, three quads of one warp per SM sub-partition, compute the column dots; the
    // quads' sums are scaled once both are done.
    const int warp = tid >> 5;
    if (warp == 0) {
        double tn0, tn1;
        if constexpr (std::is_same<T, float>::value) {
            float a0, a1;
            warp_total2<FineF32>(st.blk, 0, a0, a1);
            tn0 = a0;
            tn1 = a1;
        } else {
            warp_total2<FineF64>(st.blk, 0, tn0, tn1);
        }
        // One instruction stream for the warp: the square root of ||s'||^2 (lanes 0, 1) and of
        // ||p||^2 (lane 2) together, then 1/r_ii (the same rounded root: sigma_i is exactly
        // 1/r_ii); lane 0 keeps r_ii and the breakdown test, lane 1 sigma_i and its A::T form.
        const double y = A::round_d(sqrt(lane == 2 ? tn1 : tn0));
        const double ir = app ? A::recip_d(y) : 1.0;
        if (lane == 0) {
            const int code = !app ? 0 : (!isfinite(y) ? 1 : (!(y > 16.0 * 0x1p-53 * pref) ? 2 : 0));
            sc[0] = y;
            sc[4] = (double)code;
        } else if (lane == 1) {
            sc[1] = ir;
            sc[2] = a.p_lag ? ir : 1.0;
            const T irT = A::from_d(ir);
            scT[0] = irT;
            scT[1] = a.p_lag ? irT : A::one();
        } else if (lane == 2) {
            sc[3] = sol ? y : 0.0;
        }
    }
    if (!rich) {
        const int quad = warp / 4 - 1, qw = warp & 3;  // quads 0..2; warps 0..3 take no column
        const int seg = (k + 3) / 4;
        for (int base = 0; base < i; base += G * 3) {
            const int j = quad >= 0 ? base + blockIdx.x + G * quad : i;
            if (j < i) {
                const double* mc = st.M + (size_t)j * k;      // column i-1 was written by phase 0b
                const int l0 = qw * seg, l1 = min(k, l0 + seg);
                Acc as = A::acc0(), ap = A::acc0();
                for (int lb = l0; lb < l1; lb += 32 * 8) {   // 8 rows per lane: loads first
                    T mv[8], sv[8], pv[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const int l = lb + 32 * q + lane;
                        const bool ok = l < l1;
                        mv[q] = ok ? A::ld(mc + l) : zero;
                        sv[q] = (ok && app) ? A::ld(st.sbuf + l) : zero;
                        pv[q] = (ok && sol) ? A::ld(st.pbuf + l) : zero;
                    }
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        if (app) A::acc(as, mv[q], sv[q]);
                        if (sol) A::acc(ap, mv[q], pv[q]);
                    }
                }
                const T ds = app ? A::wsum(A::val(as)) : zero;
                const T dp = sol ? A::wsum(A::val(ap)) : zero;
                if (lane == 0) { qs[(quad * 4 + qw) * 2] = ds; qs[(quad * 4 + qw) * 2 + 1] = dp; }
            }
            __syncthreads();
            if (j < i && qw == 0 && lane == 0) {
                const T* q4 = qs + quad * 8;
                A::st(st.u2s + j, A::mul(A::add(A::add(q4[0], q4[2]), A::add(q4[4], q4[6])), scT[0]));
                A::st(st.u2p + j, A::mul(A::add(A::add(q4[1], q4[3]), A::add(q4[5], q4[7])), scT[1]));
            }
            __syncthreads();
        }
    }
    __syncthreads();                                   // warp 0's scalars, also when no column was dotted
    const double r = sc[0], pn = sc[3];
    const int code = (int)sc[4];
    const double inv_r = sc[1], pmul = sc[2];
    const T inv_rT = scT[0], pmulT = scT[1];
    if (app) {
        if (code == 1) {
            if (gtid == 0) { atomicCAS(ctl + kStatusWord, 0, (int)RGS_ERR_NONFINITE); ctl[kDetailWord] = i; }
            return;
        }
        const bool breakdown = code == 2;
        if (a.givens) {
            // GMRES: H(:, i-1) = R(0:i+1, i) (Sec. 4.1) is complete now that r_ii is known.  Its
            // rotation runs in phase 4, on a CTA without columns there while i < G, so that no
            // phase waits for it; a breakdown ends the launch here, so it runs now.
            if (i == 0) {
                if (gtid == 0) st.g[0] = r;
            } else if (breakdown && blockIdx.x == G - 1 && tid < 32) {
                givens_and_stop(st, a, r, ctl, true);
            }
        }
        if (breakdown) {
            if (!(a.arnoldi && i > 0) && gtid == 0) {
                atomicCAS(ctl + kStatusWord, 0, (int)RGS_ERR_BREAKDOWN);
                ctl[kDetailWord] = i;
            }
            return;
        }
        if (gtid == 0) {
            st.R[(size_t)i * st.ldr + i] = r;
            st.sigma[i] = inv_r;
        }
    }
    if (sol && gtid == 0) st.pnorm[a.pnorm_idx] = pn * pmul;
    if constexpr (f64) {
        if (rich) {
            richardson_phases(st, a, bar, ctl, inv_r, pmul, tr);
            return;
        }
    }
    if (!bar.sync(ctl, tr ? tr + 3 : nullptr)) return;

    // ---- phase 3: y = [s, p] - V u2 (the i reflectors applied), warp per row using the
    //      row-major copy VT; s_i is stored (step 6); sums over rows > i for the new reflector
    const int krows = app ? k : i;                 // a pure solve needs rows 0..i-1 only
    {
        Acc sg = A::acc0(), cr = A::acc0();
        for (int l = gwarp; l < krows; l += nwarps) {
            const T sl0 = app ? A::ld(st.sbuf + l) : zero;     // issued before the row's dots
            const T pl0 = sol ? A::ld(st.pbuf + l) : zero;
            T ws, wp;
            warp_row_dot2<A>(st.VT + (size_t)l * mm, st.u2s, st.u2p, min(i, l + 1), app, sol, ws, wp);
            if (lane == 0) {
                const T sl = A::mul(sl0, inv_rT);
                if (app) st.S[(size_t)i * k + l] = A::to_d(sl);      // s_i (Alg. 2 step 6)
                const T ysl = app ? A::sub(sl, ws) : zero;
                const T ypl = sol ? A::sub(A::mul(pl0, pmulT), wp) : zero;
                A::st(st.ys + l, ysl);
                A::st(st.yp + l, ypl);
                if (app && l > i) { A::acc(sg, ysl, ysl); A::acc(cr, ysl, ypl); }
            }
        }
        T sums[2] = {A::val(sg), A::val(cr)};
        block_sum_lane0<A, 2>(sums, shT);
        if (tid == 0) { A::st(st.blk + blockIdx.x * 4 + 2, sums[0]); A::st(st.blk + blockIdx.x * 4 + 3, sums[1]); }
    }
    if (!bar.sync(ctl, tr ? tr + 5 : nullptr)) return;

    if (!app) {
        // pure solve: x = R_S^{-1} y(0:i); row j of R_S^{-1} is column j of RinvT
        for (int j = gwarp; j < i; j += nwarps) {
            T d, unused;
            warp_row_dot2<A>(st.RinvT + (size_t)j * mm + j, st.yp + j, st.yp + j, i - j, true, false, d, unused);
            if (lane == 0) {
                const double dd = A::to_d(d);
                st.R[(size_t)a.xcol * st.ldr + j] = dd;
                st.coef[j] = dd * st.sigma[j];
            }
        }
        if (tr) tr[9] = globaltimer();
        return;
    }

    // The new reflector's scalars (one warp): totals SG, CR of phase 3's sums; alpha, beta, tau,
    // vs and the solve's y_i.  Warp 12 forms them at the start of phase 4 (the fourth quad has no
    // column there while i <= 3G), behind the column owners' dots.
    auto reflector_scalars = [&]() {
        T alpha = zero, ypi0 = zero;
        if (lane == 0) {                               // issued before the totals' round trip
            alpha = A::ld(st.ys + i);
            ypi0 = sol ? A::ld(st.yp + i) : zero;
        }
        T SG, CR;
        warp_total2<A>(st.blk, 2, SG, CR);
        if (lane == 0) {
            T beta, tau, vs;
            if (A::is_zero(SG)) {
                beta = alpha; tau = zero; vs = zero;
            } else {
                const T nrm = A::sqrt_(A::add(A::mul(alpha, alpha), SG));
                beta = A::nonneg(alpha) ? A::neg(nrm) : nrm;
                tau = A::div(A::sub(beta, alpha), beta);
                vs = A::div(A::one(), A::sub(alpha, beta));
            }
            scT[0] = beta; scT[1] = tau; scT[2] = vs;
            scT[3] = sol ? A::sub(ypi0, A::mul(tau, A::add(ypi0, A::mul(CR, vs)))) : zero;
        }
    };
    static_assert(NW == 16, "phase 4 runs four quads of four warps");

    // ---- phase 4 (the last): the reflector H_i, V(:, i), T(0:i, i), R_S^{-1}(:, i) and x.  Per
    //   column j < i, by the four warps of one quad: T(j, i) = -tau (a_j + vs b_j) with
    //   a_j = sum_{j<=l<i} T(j,l) V(i,l) and b_j = sum_{l>i} N(l,j) ys_l (N = V T^T, kept by phase
    //   0: b_j = sum_l T(j,l) zp_l with zp_l = sum_{r>i} V(r,l) ys_r, the same sum in the other
    //   order, so no grid phase waits for the zp), and d1_j = sum_{j<=l<i} Rinv(j,l) ys_l (d2_j
    //   likewise with yp) for R_S^{-1}(j, i) = -d1_j / beta and x_j; the quad's lane 0 finishes
    //   the column.  GMRES: warp 0 of the last CTA rotates H(:, i-1).
    if (a.givens && i > 0 && blockIdx.x == G - 1 && tid < 32) givens_and_stop(st, a, r, ctl, false);
    if (warp == 12) reflector_scalars();               // read after the quads' first barrier
    {
        // quad 3 splits its column over warps 13..15: warp 12 forms the scalars (and adds zeros)
        const int quad = tid >> 7, qw = (tid >> 5) & 3;
        const int nq = quad == 3 ? 3 : 4, qi = quad == 3 ? qw - 1 : qw;
        const double* vrow_i = st.VT + (size_t)i * mm;     // V(i, 0:i)
        for (int base = 0; base < i; base += G * (NW / 4)) {
            const int j = base + blockIdx.x + G * quad;
            if (j < i && qi < 0 && lane == 0) {
                qs[(quad * 4 + qw) * 3] = zero;
                qs[(quad * 4 + qw) * 3 + 1] = zero;
                qs[(quad * 4 + qw) * 3 + 2] = zero;
                shT[quad * 4 + qw] = zero;
            } else if (j < i && qi >= 0) {
                const double* nc = st.N + (size_t)j * k;
                const int len = k - (i + 1), seg = (max(len, 0) + nq - 1) / nq;
                const int l0 = i + 1 + qi * seg, l1 = min(k, l0 + seg);
                Acc ab = A::acc0(), aa = A::acc0(), a1 = A::acc0(), a2 = A::acc0();
                for (int lb = l0; lb < l1; lb += 32 * 8) {   // loads of 8 rows per lane first
                    T nv[8], yv[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const int l = lb + 32 * q + lane;
                        nv[q] = l < l1 ? A::ldcg(nc + l) : zero;    // N is written in this launch
                        yv[q] = l < l1 ? A::ld(st.ys + l) : zero;
                    }
#pragma unroll
                    for (int q = 0; q < 8; ++q) A::acc(ab, nv[q], yv[q]);
                }
                const double* rr = st.RinvT + (size_t)j * mm;       // row j of R_S^{-1}
                const double* tt = st.TT + (size_t)j * mm;          // row j of T
                const int rlen = i - j, rseg = (rlen + nq - 1) / nq;
                const int r0 = j + qi * rseg, r1 = min(i, r0 + rseg);
                for (int lb = r0; lb < r1; lb += 32 * 4) {
                    T rv[4], y1[4], y2[4], tv[4], vv[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int l = lb + 32 * q + lane;
                        const bool ok = l < r1;
                        rv[q] = ok ? A::ld(rr + l) : zero;
                        y1[q] = ok ? A::ld(st.ys + l) : zero;
                        y2[q] = (ok && sol) ? A::ld(st.yp + l) : zero;
                        tv[q] = ok ? A::ld(tt + l) : zero;
                        vv[q] = ok ? A::ld(vrow_i + l) : zero;
                    }
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        A::acc(a1, rv[q], y1[q]);
                        if (sol) A::acc(a2, rv[q], y2[q]);
                        A::acc(aa, tv[q], vv[q]);
                    }
                }
                const T bsum = A::wsum(A::val(ab));
                const T asum = A::wsum(A::val(aa));
                const T d1 = A::wsum(A::val(a1));
                const T d2 = sol ? A::wsum(A::val(a2)) : zero;
                if (lane == 0) {
                    qs[(quad * 4 + qw) * 3] = bsum;
                    qs[(quad * 4 + qw) * 3 + 1] = d1;
                    qs[(quad * 4 + qw) * 3 + 2] = d2;
                    shT[quad * 4 + qw] = asum;
                }
            }
            __syncthreads();
            const T beta = scT[0], tau = scT[1], vs = scT[2], ypi = scT[3];
            if (j < i && qw == 0 && lane == 0 && !A::is_zero(beta)) {   // column j's entries of T, R_S^{-1}, x
                const T* q4 = qs + quad * 12;
                const T bj = A::add(A::add(q4[0], q4[3]), A::add(q4[6], q4[9]));
                const T d1j = A::add(A::add(q4[1], q4[4]), A::add(q4[7], q4[10]));
                const T d2j = A::add(A::add(q4[2], q4[5]), A::add(q4[8], q4[11]));
                const T* s4 = shT + quad * 4;
                const T aj = A::add(A::add(s4[0], s4[1]), A::add(s4[2], s4[3]));
                const T t = A::neg(A::mul(tau, A::add(aj, A::mul(vs, bj))));
                A::st(st.T + (size_t)i * mm + j, t);
                A::st(st.TT + (size_t)j * mm + i, t);
                const T cnew = A::neg(A::div(d1j, beta));            // R_S^{-1}(j, i)
                A::st(st.RinvT + (size_t)j * mm + i, cnew);
                if (sol) {
                    const double xj = A::to_d(A::add(d2j, A::mul(cnew, ypi)));
                    st.R[(size_t)a.xcol * st.ldr + j] = xj;
                    st.coef[j] = xj * st.sigma[j];
                }
            }
            __syncthreads();
        }
    }
    __syncthreads();                                   // the scalars, also when no column was done
    const T beta = scT[0], tau = scT[1], vs = scT[2], ypi = scT[3];
    if (A::is_zero(beta)) {
        if (gtid == 0) { atomicCAS(ctl + kStatusWord, 0, (int)RGS_ERR_BREAKDOWN); ctl[kDetailWord] = i; }
        return;
    }
    for (int l = gtid; l < k; l += nthreads) {
        const T vl = l < i ? zero : (l == i ? A::one() : A::mul(A::ld(st.ys + l), vs));
        A::st(st.V + (size_t)i * k + l, vl);
        if (l >= i) A::st(st.VT + (size_t)l * mm + i, vl);
    }
    if (gtid == 0) {
        A::st(st.T + (size_t)i * mm + i, tau);
        A::st(st.TT + (size_t)i * mm + i, tau);
        A::st(st.RinvT + (size_t)i * mm + i, A::div(A::one(), beta));
        if (sol) {
            const double xi = A::to_d(A::div(ypi, beta));
            st.R[(size_t)a.xcol * st.ldr + i] = xi;
            st.coef[i] = xi * inv_r;
        }
    }
    if (tr) tr[9] = globaltimer();
}


// Step 8 certificates: Delta_m = ||I - S^T S||_F, Delta~_m = ||P - S R||_F / ||P||_F.
// Block t handles the columns b = t and b = m-1-t (equal total work per block): the entries
// (I - S^T S)(a, b) for a <= b (the matrix is symmetric, so the off-diagonal squares count twice)
// and the column (P - S R)(:, b), accumulated as sums of squares.
__global__ void __launch_bounds__(256) cert_kernel(const double* S, int k, int m, const double* R, int64_t ldr,
                                                   const double* P, double* work) {
    __shared__ double sh[256];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    double g2 = 0.0, e2 = 0.0, p2 = 0.0;
    const int t = blockIdx.x;
    for (int h = 0; h < 2; ++h) {
        const int b = h == 0 ? t : m - 1 - t;
        if (h == 1 && b == t) break;
        for (int a = w; a <= b; a += 8) {
            double d = 0.0;
            for (int l = lane; l < k; l += 32) d = fma(S[(size_t)a * k + l], S[(size_t)b * k + l], d);
            d = warp_sum(d);
            const double e = (a == b ? 1.0 : 0.0) - d;
            g2 += lane == 0 ? (a == b ? e * e : 2.0 * (e * e)) : 0.0;
        }
        for (int l = threadIdx.x; l < k; l += 256) {
            double v = P[(size_t)b * k + l];
            p2 += v * v;
            for (int j = 0; j <= b; ++j) v = fma(-S[(size_t)j * k + l], R[(size_t)b * ldr + j], v);
            e2 += v * v;
        }
    }
    g2 = block_sum<256>(g2, sh);
    e2 = block_sum<256>(e2, sh);
    p2 = block_sum<256>(p2, sh);
    if (threadIdx.x == 0) { work[3 * t] = g2; work[3 * t + 1] = e2; work[3 * t + 2] = p2; }
}

__global__ void cert_final_kernel(const double* work, int m, double* out) {
    __shared__ double sh[256];
    double g = 0.0, e = 0.0, p = 0.0;
    for (int b = threadIdx.x; b < m; b += 256) { g += work[3 * b]; e += work[3 * b + 1]; p += work[3 * b + 2]; }
    g = block_sum<256>(g, sh);
    e = block_sum<256>(e, sh);
    p = block_sum<256>(p, sh);
    if (threadIdx.x == 0) { out[0] = sqrt(g); out[1] = sqrt(e / p); }
}

}  // namespace

void rgs_ls_alloc(DevBuf& buf, int k, int mmax, int grid, int max_parts, int fine_df, LSState* st) {
    size_t n = 0;
    auto take = [&](size_t cnt) { size_t off = n; n += (cnt + 31) & ~(size_t)31; return off; };
    const size_t oV = take((size_t)k * mmax), oVT = take((size_t)k * mmax), oT = take((size_t)mmax * mmax),
                 oTT = take((size_t)mmax * mmax), oRi = take((size_t)mmax * mmax), oS = take((size_t)k * mmax),
                 osb = take(k), opb = take(k), oys = take(k), oyp = take(k), oM = take((size_t)k * mmax),
                 ou2s = take(mmax), ou2p = take(mmax), oN = take((size_t)k * mmax), onf = take(1),
                 od1 = take(mmax), od2 = take(mmax),
                 oblk = take((size_t)4 * grid), osg = take(mmax + 1),
                 opn = take(mmax + 2), oco = take(mmax + 1);
    buf.ensure(n * sizeof(double));
    double* b = buf.as<double>();
    st->k = k; st->mmax = mmax; st->max_parts = max_parts; st->fine_df = fine_df;
    st->V = b + oV; st->VT = b + oVT; st->T = b + oT; st->TT = b + oTT; st->RinvT = b + oRi; st->S = b + oS;
    st->sbuf = b + osb; st->pbuf = b + opb; st->ys = b + oys; st->yp = b + oyp;
    st->M = b + oM; st->u2s = b + ou2s; st->u2p = b + ou2p;
    st->N = b + oN; st->nfold = reinterpret_cast<int*>(b + onf); st->d1 = b + od1; st->d2 = b + od2;
    st->blk = b + oblk; st->sigma = b + osg; st->pnorm = b + opn;
    st->coef = b + oco;
}

// Zero the factorisation (V must be zero above each reflector's diagonal; T, R_S^{-1} upper parts).
void rgs_ls_reset(rgs_context* ctx, const LSState& st) {
    RGS_CUDA(cudaMemsetAsync(st.V, 0, sizeof(double) * (size_t)st.k * st.mmax, ctx->stream));
    RGS_CUDA(cudaMemsetAsync(st.VT, 0, sizeof(double) * (size_t)st.k * st.mmax, ctx->stream));
    RGS_CUDA(cudaMemsetAsync(st.T, 0, sizeof(double) * (size_t)st.mmax * st.mmax, ctx->stream));
    RGS_CUDA(cudaMemsetAsync(st.TT, 0, sizeof(double) * (size_t)st.mmax * st.mmax, ctx->stream));
    RGS_CUDA(cudaMemsetAsync(st.RinvT, 0, sizeof(double) * (size_t)st.mmax * st.mmax, ctx->stream));
    RGS_CUDA(cudaMemsetAsync(st.pnorm, 0, sizeof(double) * (size_t)(st.mmax + 2), ctx->stream));
    RGS_CUDA(cudaMemsetAsync(st.nfold, 0, sizeof(int), ctx->stream));
}

int rgs_ls_grid(const rgs_context* ctx) {
    return ctx->ls_blocks_tuned > 0 ? std::min(ctx->ls_blocks_tuned, ctx->ls_blocks) : ctx->ls_blocks;
}

const void* ls_kernel_for(int fine_df) {
    return fine_df == 2 ? (const void*)ls_kernel<FineF32>
           : fine_df ? (const void*)ls_kernel<FineDF> : (const void*)ls_kernel<FineF64>;
}

void rgs_launch_ls(rgs_context* ctx, const LSState& st, const LSStep& a) {
    RGS_REQUIRE(a.s_nparts <= st.max_parts && a.p_nparts <= st.max_parts, "too many partial sketches");
    LSState s = st;
    LSStep p = a;
    void* args[] = {&s, &p};
    const int grid = rgs_ls_grid(ctx);
    RGS_REQUIRE(grid <= 32 * kTotMax, "least-squares grid larger than the per-CTA totals support");
    const void* fn = ls_kernel_for(st.fine_df);
    cudaLaunchAttribute attrs[2] = {};
    attrs[0].id = cudaLaunchAttributeCooperative;
    attrs[0].val.cooperative = 1;
    attrs[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attrs[1].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(LT);
    cfg.stream = ctx->stream;
    cfg.attrs = attrs;
    cfg.numAttrs = (ctx->pdl && ctx->pdl_coop) ? 2 : 1;
    cudaError_t e = cudaLaunchKernelExC(&cfg, fn, args);
    if (e != cudaSuccess && cfg.numAttrs == 2) {
        // the driver refused programmatic serialization with a cooperative launch: plain order
        cudaGetLastError();
        ctx->pdl_coop = 0;
        cfg.numAttrs = 1;
        e = cudaLaunchKernelExC(&cfg, fn, args);
    }
    RGS_CUDA(e);
    ctx->launches++;
}

// One CTA of LT threads per SM (its registers fill the SM), so the cooperative grid is the SM count.
int rgs_ls_max_blocks(int num_sms) {
    for (int f = 0; f < 3; ++f) {
        const void* fn = ls_kernel_for(f);
        int per_sm = 0;
        RGS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, LT, 0));
        RGS_REQUIRE(per_sm >= 1, "the least-squares kernel does not fit on an SM");
    }
    return num_sms;
}

void rgs_launch_certificates(rgs_context* ctx, const double* S, int k, int m, const double* R, int64_t ldr,
                             const double* P, double* out2, double* work) {
    const int nb = (m + 1) / 2;                     // block t: columns t and m-1-t
    cert_kernel<<<nb, 256, 0, ctx->stream>>>(S, k, m, R, ldr, P, work);
    RGS_CUDA(cudaGetLastError());
    cert_final_kernel<<<1, 256, 0, ctx->stream>>>(work, nb, out2);
    RGS_CUDA(cudaGetLastError());
    ctx->launches += 2;
}
