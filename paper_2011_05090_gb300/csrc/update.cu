// Fused RGS step 3 + step 4 (Alg. 2): q'_i = w_i - Q'_{i-1} c, rounded to the
// storage type and written once, then sketched from the stored values without
// re-reading them.  The SRHT sketch is applied per tile of 1024 rows: signs,
// an in-register / warp-shuffle / shared-memory Walsh-Hadamard transform of
// the tile, and the tile's contribution to each sampled output row
// (H_s = H_{s/1024} (x) H_1024, so output row a*1024+b gets
// (-1)^popcount(a & t) * (H_1024 z_t)[b] from tile t).  Per-CTA partial
// k-vectors are summed later in a fixed order (deterministic).
#include "fwht.cuh"

#include <algorithm>
#include <type_traits>

using namespace rgsdev;

namespace {

constexpr int UT = TILE_THREADS;   // threads per CTA, 4 consecutive rows each
constexpr int UNROLL = 8;    // basis columns loaded ahead

// Streaming loads of the basis and of w: they are read once per column step and would
// otherwise evict the least-squares factors (V, T, S: a few tens of MB) from L2.
__device__ __forceinline__ uint64_t evict_first_policy() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ float4 ld_stream_f4(const void* p, uint64_t pol) {
    float4 v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.f32 {%0,%1,%2,%3}, [%4], %5;"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ double2 ld_stream_d2(const void* p, uint64_t pol) {
    double2 v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.f64 {%0,%1}, [%2], %3;"
                 : "=d"(v.x), "=d"(v.y)
                 : "l"(p), "l"(pol));
    return v;
}
__device__ __forceinline__ uint2 ld_stream_u2(const void* p, uint64_t pol) {
    uint2 v;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.u32 {%0,%1}, [%2], %3;"
                 : "=r"(v.x), "=r"(v.y)
                 : "l"(p), "l"(pol));
    return v;
}

template <typename TQ> struct QIO;

template <> struct QIO<double> {
    using Acc = double;
    __device__ static void load4(const double* p, double v[4], uint64_t pol) {
        double2 a = ld_stream_d2(p, pol);
        double2 b = ld_stream_d2(p + 2, pol);
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
    __device__ static void store4(double* p, const double v[4]) {
        reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
        reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
    }
    __device__ static double load1(const double* p) { return __ldg(p); }
    __device__ static void store1(double* p, double v) { *p = v; }
    __device__ static double to_storage(double v) { return v; }
};

template <> struct QIO<float> {
    using Acc = float;
    __device__ static void load4(const float* p, float v[4], uint64_t pol) {
        float4 a = ld_stream_f4(p, pol);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    }
    __device__ static void store4(float* p, const float v[4]) {
        *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    }
    __device__ static float load1(const float* p) { return __ldg(p); }
    __device__ static void store1(float* p, float v) { *p = v; }
    __device__ static float to_storage(float v) { return v; }
};

template <> struct QIO<__nv_bfloat16> {
    using Acc = float;
    __device__ static void load4(const __nv_bfloat16* p, float v[4], uint64_t pol) {
        uint2 a = ld_stream_u2(p, pol);
        __nv_bfloat162 x = *reinterpret_cast<__nv_bfloat162*>(&a.x);
        __nv_bfloat162 y = *reinterpret_cast<__nv_bfloat162*>(&a.y);
        float2 fx = __bfloat1622float2(x), fy = __bfloat1622float2(y);
        v[0] = fx.x; v[1] = fx.y; v[2] = fy.x; v[3] = fy.y;
    }
    __device__ static void store4(__nv_bfloat16* p, const float v[4]) {
        __nv_bfloat162 x = __floats2bfloat162_rn(v[0], v[1]);
        __nv_bfloat162 y = __floats2bfloat162_rn(v[2], v[3]);
        uint2 a;
        a.x = *reinterpret_cast<uint32_t*>(&x);
        a.y = *reinterpret_cast<uint32_t*>(&y);
        *reinterpret_cast<uint2*>(p) = a;
    }
    __device__ static float load1(const __nv_bfloat16* p) { return __bfloat162float(p[0]); }
    __device__ static void store1(__nv_bfloat16* p, float v) { p[0] = __float2bfloat16_rn(v); }
    // value actually stored, back in float
    __device__ static float to_storage(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }
};

struct UpdParams {
    int64_t n;
    int ncols;
    const void* Q;
    int64_t ldq;
    const double* w;
    int64_t ldw;
    const double* wscale;
    int w_df;                 // w holds double-float pairs (float2) instead of FP64
    const double* coef;
    void* qout;
    const double* w_next;     // blockIdx.y == 1 sketches this FP64 column (no update, no store)
    const uint32_t* signbits;
    const int32_t* rows;
    int k;
    int ntiles;
    int vec;
    double* partials;
    const int* ctl;
};

// FM: arithmetic of the transform sums: 0 FP64, 1 double-float, 2 FP32 (partials written as
// double-float pairs with a zero low word, the layout the least-squares kernel reads).
template <typename TQ, bool SRHT, int FM>
__global__ void __launch_bounds__(UT, 4) update_sketch_kernel(UpdParams p) {
    using IO = QIO<TQ>;
    using Acc = typename IO::Acc;
    using V = typename std::conditional<FM == 1, df, typename std::conditional<FM == 2, float, double>::type>::type;
    using F = FW<V>;
    extern __shared__ __align__(16) double smem[];
    V* zt = reinterpret_cast<V*>(smem);                  // TILE
    V* part = zt + TILE;                                 // k
    int32_t* srow = reinterpret_cast<int32_t*>(part + (SRHT ? p.k : 0));     // k
    Acc* sc = reinterpret_cast<Acc*>(srow + (SRHT ? ((p.k + 3) & ~3) : 0));   // ncols

    pdl_wait();                        // the previous kernel's coefficients, status and basis
    pdl_launch_dependents();
    if (p.ctl != nullptr && p.ctl[kStatusWord] != 0) return;   // an earlier step failed or broke down
    const int col = blockIdx.y;
    // the second row of blocks of a launch with w_next sketches the next input column as it is
    // (Alg. 2 step 1 of column i + 1, in FP64 / double-float) while the first updates column i
    const bool next_role = p.w_next != nullptr && col == 1;
    const double* w = next_role ? p.w_next : p.w + (int64_t)col * p.ldw;
    const double wmul = p.wscale ? *p.wscale : 1.0;
    const TQ* Q = reinterpret_cast<const TQ*>(p.Q);
    TQ* qout = reinterpret_cast<TQ*>(p.qout);
    const int64_t n = p.n;
    const uint64_t pol = evict_first_policy();

    for (int j = threadIdx.x; j < p.ncols; j += UT) sc[j] = (Acc)p.coef[j];
    if (SRHT)
        for (int j = threadIdx.x; j < p.k; j += UT) { srow[j] = p.rows[j]; part[j] = F::zero(); }
    __syncthreads();

    for (int tile = blockIdx.x; tile < p.ntiles; tile += gridDim.x) {
        const int64_t r0 = (int64_t)tile * TILE + threadIdx.x * 4;
        const bool full = p.vec && (r0 + 4 <= n);
        if (SRHT && next_role) {
            V z[4];
            if (full) {
                const double2 a = ld_stream_d2(w + r0, pol), b = ld_stream_d2(w + r0 + 2, pol);
                z[0] = F::from(a.x); z[1] = F::from(a.y); z[2] = F::from(b.x); z[3] = F::from(b.y);
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e) z[e] = F::from(r0 + e < n ? w[r0 + e] : 0.0);
            }
            srht_tile<V>(z, r0, n, tile, p.signbits, srow, p.k, zt, part);
            continue;
        }
        Acc acc[4];
        if (full) {
            if (p.w_df) {            // hi + lo rounded once to the accumulation type
                const float4 a = ld_stream_f4(w + r0, pol), b = ld_stream_f4(w + r0 + 2, pol);
                if constexpr (sizeof(Acc) == 4) {
                    acc[0] = a.x + a.y; acc[1] = a.z + a.w; acc[2] = b.x + b.y; acc[3] = b.z + b.w;
                    if (p.wscale) {
                        const float fm = (float)wmul;
#pragma unroll
                        for (int e = 0; e < 4; ++e) acc[e] *= fm;
                    }
                } else {
                    acc[0] = (double)a.x + (double)a.y; acc[1] = (double)a.z + (double)a.w;
                    acc[2] = (double)b.x + (double)b.y; acc[3] = (double)b.z + (double)b.w;
                    if (p.wscale)
#pragma unroll
                        for (int e = 0; e < 4; ++e) acc[e] *= wmul;
                }
            } else {
                double2 a = ld_stream_d2(w + r0, pol);
                double2 b = ld_stream_d2(w + r0 + 2, pol);
                if (p.wscale) { a.x *= wmul; a.y *= wmul; b.x *= wmul; b.y *= wmul; }
                acc[0] = (Acc)a.x; acc[1] = (Acc)a.y; acc[2] = (Acc)b.x; acc[3] = (Acc)b.y;
            }
            int j = 0;
            for (; j + UNROLL <= p.ncols; j += UNROLL) {
                Acc q[UNROLL][4];
#pragma unroll
                for (int u = 0; u < UNROLL; ++u) IO::load4(Q + (int64_t)(j + u) * p.ldq + r0, q[u], pol);
#pragma unroll
                for (int u = 0; u < UNROLL; ++u) {
                    const Acc c = sc[j + u];
#pragma unroll
                    for (int e = 0; e < 4; ++e) acc[e] = fma(-c, q[u][e], acc[e]);
                }
            }
            for (; j < p.ncols; ++j) {
                Acc q[4];
                IO::load4(Q + (int64_t)j * p.ldq + r0, q, pol);
                const Acc c = sc[j];
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[e] = fma(-c, q[e], acc[e]);
            }
        } else {
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                if (r0 + e >= n) { acc[e] = (Acc)0; continue; }
                if (p.w_df) {
                    const float2 d = reinterpret_cast<const float2*>(w)[r0 + e];
                    if constexpr (sizeof(Acc) == 4) acc[e] = (d.x + d.y) * (float)wmul;
                    else acc[e] = (Acc)(((double)d.x + (double)d.y) * wmul);
                } else {
                    acc[e] = (Acc)(w[r0 + e] * wmul);
                }
            }
            for (int j = 0; j < p.ncols; ++j) {
                const Acc c = sc[j];
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (r0 + e < n) acc[e] = fma(-c, IO::load1(Q + (int64_t)j * p.ldq + r0 + e), acc[e]);
            }
        }
        V z[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            acc[e] = IO::to_storage(acc[e]);
            if constexpr (sizeof(Acc) == 4) z[e] = F::from_float((r0 + e < n) ? (float)acc[e] : 0.f);
            else z[e] = F::from((r0 + e < n) ? (double)acc[e] : 0.0);
        }
        if (qout != nullptr) {
            if (full) {
                IO::store4(qout + r0, acc);
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (r0 + e < n) IO::store1(qout + r0 + e, acc[e]);
            }
        }
        if (SRHT) srht_tile<V>(z, r0, n, tile, p.signbits, srow, p.k, zt, part);
    }
    if (SRHT) {
        __syncthreads();
        const int64_t o = ((int64_t)col * gridDim.x + blockIdx.x) * p.k;
        if constexpr (FM == 2) {
            df* out = reinterpret_cast<df*>(p.partials) + o;
            for (int j = threadIdx.x; j < p.k; j += UT) out[j] = df{part[j], 0.f};
        } else {
            V* out = reinterpret_cast<V*>(p.partials) + o;
            for (int j = threadIdx.x; j < p.k; j += UT) out[j] = part[j];
        }
    }
}

// Gaussian sketch partials: partial_b = Theta[:, rows of block b] x[rows of block b].
template <typename TX>
__global__ void __launch_bounds__(256) gauss_sketch_kernel(const double* __restrict__ theta, int k, int64_t n,
                                                           const TX* __restrict__ x, int64_t ldx,
                                                           double* __restrict__ partials, const int* ctl) {
    constexpr int CH = 256;
    __shared__ double xs[CH];
    if (ctl != nullptr && ctl[kStatusWord] != 0) return;
    const int col = blockIdx.y;
    x += (int64_t)col * ldx;
    const int64_t per = (n + gridDim.x - 1) / gridDim.x;
    const int64_t c0 = (int64_t)blockIdx.x * per;
    const int64_t c1 = min(n, c0 + per);
    double* out = partials + ((int64_t)col * gridDim.x + blockIdx.x) * k;
    for (int lb = 0; lb < k; lb += 1024) {           // rows lb + threadIdx.x + 256 t of Theta
        double acc[4] = {0.0, 0.0, 0.0, 0.0};
        for (int64_t cb = c0; cb < c1; cb += CH) {
            const int len = (int)min((int64_t)CH, c1 - cb);
            __syncthreads();
            if (threadIdx.x < len) {
                if constexpr (sizeof(TX) == 2) xs[threadIdx.x] = (double)__bfloat162float(x[cb + threadIdx.x]);
                else xs[threadIdx.x] = (double)x[cb + threadIdx.x];
            }
            __syncthreads();
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int l = lb + threadIdx.x + 256 * t;
                if (l < k) {
                    const double* th = theta + cb * k + l;
                    double a = acc[t];
                    for (int c = 0; c < len; ++c) a = fma(__ldg(th + (int64_t)c * k), xs[c], a);
                    acc[t] = a;
                }
            }
        }
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int l = lb + threadIdx.x + 256 * t;
            if (l < k) out[l] = acc[t];
        }
    }
}

// Two columns in one pass over Theta (the one-synchronisation RGS-Arnoldi of Sec. 2.4 with a
// Gaussian sketch: Theta q'_i and Theta A q'_i are formed together, a two-column product, instead
// of reading the k x n matrix once per vector).  Rows, blocks and the order of every sum are those
// of gauss_sketch_kernel, so each column's partials are bit-identical to a one-column launch.
template <typename TX>
__global__ void __launch_bounds__(256) gauss_sketch2_kernel(const double* __restrict__ theta, int k, int64_t n,
                                                            const TX* __restrict__ x1, const double* __restrict__ x2,
                                                            double* __restrict__ part1, double* __restrict__ part2,
                                                            const int* ctl) {
    constexpr int CH = 256;
    __shared__ double xs1[CH], xs2[CH];
    if (ctl != nullptr && ctl[kStatusWord] != 0) return;
    const int64_t per = (n + gridDim.x - 1) / gridDim.x;
    const int64_t c0 = (int64_t)blockIdx.x * per;
    const int64_t c1 = min(n, c0 + per);
    double* o1 = part1 + (int64_t)blockIdx.x * k;
    double* o2 = part2 + (int64_t)blockIdx.x * k;
    for (int lb = 0; lb < k; lb += 1024) {
        double a1[4] = {0.0, 0.0, 0.0, 0.0}, a2[4] = {0.0, 0.0, 0.0, 0.0};
        for (int64_t cb = c0; cb < c1; cb += CH) {
            const int len = (int)min((int64_t)CH, c1 - cb);
            __syncthreads();
            if (threadIdx.x < len) {
                if constexpr (sizeof(TX) == 2) xs1[threadIdx.x] = (double)__bfloat162float(x1[cb + threadIdx.x]);
                else xs1[threadIdx.x] = (double)x1[cb + threadIdx.x];
                xs2[threadIdx.x] = x2[cb + threadIdx.x];
            }
            __syncthreads();
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const int l = lb + threadIdx.x + 256 * t;
                if (l < k) {
                    const double* th = theta + cb * k + l;
                    double u = a1[t], v = a2[t];
                    for (int c = 0; c < len; ++c) {
                        const double tc = __ldg(th + (int64_t)c * k);
                        u = fma(tc, xs1[c], u);
                        v = fma(tc, xs2[c], v);
                    }
                    a1[t] = u;
                    a2[t] = v;
                }
            }
        }
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int l = lb + threadIdx.x + 256 * t;
            if (l < k) {
                o1[l] = a1[t];
                o2[l] = a2[t];
            }
        }
    }
}

template <bool DF>
__global__ void reduce_partials_kernel(const double* __restrict__ partials, int nparts, int k, double scale,
                                       double* __restrict__ Y, int64_t ldy) {
    const int col = blockIdx.y;
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= k) return;
    double v;
    if constexpr (DF) {
        const df* src = reinterpret_cast<const df*>(partials) + (int64_t)col * nparts * k + l;
        df t = {0.f, 0.f};
        for (int b = 0; b < nparts; ++b) t = df_add(t, src[(int64_t)b * k]);
        v = (double)t.h + (double)t.l;
    } else {
        const double* src = partials + (int64_t)col * nparts * k + l;
        v = 0.0;
        for (int b = 0; b < nparts; ++b) v += src[(int64_t)b * k];
    }
    Y[(int64_t)col * ldy + l] = v * scale;
}

__global__ void gaussian_theta_kernel(double* theta, int k, int64_t n, uint32_t key0, uint32_t key1) {
    const int pairs = (k + 1) / 2;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)pairs * n) return;
    const int64_t c = idx / pairs;
    const int pr = (int)(idx - c * pairs);
    uint32_t ctr[4] = {(uint32_t)c, (uint32_t)pr, 0u, 0u};
    philox4x32_10(ctr, key0, key1);
    const double u1 = u53(ctr[0], ctr[1]), u2 = u53(ctr[2], ctr[3]);
    const double rad = sqrt(-2.0 * log(u1));
    double sn, cs;
    sincos(2.0 * M_PI * u2, &sn, &cs);
    const double scale = 1.0 / sqrt((double)k);
    theta[c * k + 2 * pr] = rad * cs * scale;
    if (2 * pr + 1 < k) theta[c * k + 2 * pr + 1] = rad * sn * scale;
}

template <typename TQ, bool SRHT, int FM = 0>
void launch_update_t(rgs_context* ctx, const UpdParams& p, int gx, int gy, size_t smem) {
    auto kern = update_sketch_kernel<TQ, SRHT, FM>;
    if (smem > 48 * 1024) RGS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    cudaLaunchAttribute attr{};
    attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr.val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(gx, gy);
    cfg.blockDim = dim3(UT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = ctx->stream;
    cfg.attrs = &attr;
    cfg.numAttrs = ctx->pdl ? 1 : 0;
    RGS_CUDA(cudaLaunchKernelEx(&cfg, kern, p));
    ctx->launches++;
}

template <typename TX>
void launch_gauss_t(rgs_context* ctx, const double* theta, int k, int64_t n, const void* x, int64_t ldx, int cols,
                    double* partials, int gx, const int* ctl) {
    gauss_sketch_kernel<TX><<<dim3(gx, cols), 256, 0, ctx->stream>>>(theta, k, n, reinterpret_cast<const TX*>(x),
                                                                       ldx, partials, ctl);
    RGS_CUDA(cudaGetLastError());
    ctx->launches++;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

int rgs_update_nparts(const rgs_context* ctx, const rgs_sketch_obj* sk, int64_t n, int wcols) {
    const int ntiles = (int)((n + TILE - 1) / TILE);
    if (sk->kind != RGS_SKETCH_SRHT) return std::max(1, std::min((int)((n + 255) / 256), ctx->num_sms * 2));
    const int slots = ctx->num_sms * std::min(ctx->upd_blocks_per_sm, kUpdMaxBlocksPerSm);
    if (wcols <= 1) return std::max(1, std::min(ntiles, slots));
    return std::max(1, std::min(ntiles, std::max(4, 8 * slots / wcols)));
}

// Launch the fused update (optional) + sketch.  Writes partial sketches for each
// input column to `partials` ([col][nparts][k]) and returns nparts through *nparts.
int rgs_launch_update_sketch(rgs_context* ctx, const rgs_sketch_obj* sk, const UpdateLaunch& L, double* partials,
                             int* nparts, const int* ctl) {
    const int64_t n = L.n;
    const int ntiles = (int)((n + TILE - 1) / TILE);
    const size_t esz = L.qtype == RGS_F64 ? 8 : (L.qtype == RGS_F32 ? 4 : 2);
    UpdParams p{};
    p.n = n;
    p.ncols = L.ncols;
    p.Q = L.Q;
    p.ldq = L.ldq;
    p.w = L.w;
    p.ldw = L.ldw;
    p.wscale = L.wscale;
    p.w_df = L.w_df;
    p.coef = L.coef;
    p.qout = L.qout;
    p.w_next = L.w_next;
    p.ntiles = ntiles;
    p.ctl = ctl;
    p.k = sk->k;
    // vector path: every 4-row group of w, Q and q_out starts on a 16-byte (bf16: 8-byte) boundary
    RGS_REQUIRE(L.w_next == nullptr || (L.wcols == 1 && sk->kind == RGS_SKETCH_SRHT),
                "a fused next-column sketch needs one input column and an SRHT sketch");
    bool vec = aligned16(L.w) && (L.wcols == 1 || L.ldw % 2 == 0);
    if (L.w_next) vec = vec && aligned16(L.w_next);
    if (L.ncols > 0) vec = vec && aligned16(L.Q) && (L.ldq % 4 == 0);
    if (L.qout) vec = vec && ((uintptr_t)L.qout % (4 * esz) == 0 || aligned16(L.qout)) && (L.ldq % 4 == 0);
    p.vec = vec ? 1 : 0;
    const bool srht = sk->kind == RGS_SKETCH_SRHT;
    int gx = srht ? rgs_update_nparts(ctx, sk, n, L.wcols)
                  : std::max(1, std::min(ntiles, ctx->num_sms * std::min(ctx->upd_blocks_per_sm, kUpdMaxBlocksPerSm)));
    if (srht && L.max_parts > 0) gx = std::min(gx, L.max_parts);
    if (srht) {
        p.signbits = sk->signbits.as<uint32_t>();
        p.rows = sk->rows.as<int32_t>();
        p.partials = partials;
    }
    size_t accsz = (L.qtype == RGS_F64) ? 8 : 4;
    size_t smem = TILE * 8 + (srht ? (size_t)p.k * 8 + (size_t)((p.k + 3) & ~3) * 4 : 0) + (size_t)L.ncols * accsz + 16;
    if (L.ncols > 0 || L.qout || srht) {
        const int gy = L.w_next ? 2 : L.wcols;
        if (srht && L.df_sketch == 2) {
            switch (L.qtype) {
                case RGS_F64: launch_update_t<double, true, 2>(ctx, p, gx, gy, smem); break;
                case RGS_F32: launch_update_t<float, true, 2>(ctx, p, gx, gy, smem); break;
                default: launch_update_t<__nv_bfloat16, true, 2>(ctx, p, gx, gy, smem); break;
            }
        } else if (srht && L.df_sketch) {
            switch (L.qtype) {
                case RGS_F64: launch_update_t<double, true, 1>(ctx, p, gx, gy, smem); break;
                case RGS_F32: launch_update_t<float, true, 1>(ctx, p, gx, gy, smem); break;
                default: launch_update_t<__nv_bfloat16, true, 1>(ctx, p, gx, gy, smem); break;
            }
        } else if (srht) {
            switch (L.qtype) {
                case RGS_F64: launch_update_t<double, true>(ctx, p, gx, gy, smem); break;
                case RGS_F32: launch_update_t<float, true>(ctx, p, gx, gy, smem); break;
                default: launch_update_t<__nv_bfloat16, true>(ctx, p, gx, gy, smem); break;
            }
        } else {
            switch (L.qtype) {
                case RGS_F64: launch_update_t<double, false>(ctx, p, gx, gy, smem); break;
                case RGS_F32: launch_update_t<float, false>(ctx, p, gx, gy, smem); break;
                default: launch_update_t<__nv_bfloat16, false>(ctx, p, gx, gy, smem); break;
            }
        }
    }
    if (srht) {
        *nparts = gx;
        return gx;
    }
    // Gaussian: sketch the stored column (or the input columns when nothing is stored)
    int gg = rgs_update_nparts(ctx, sk, n, L.wcols);
    if (L.max_parts > 0) gg = std::min(gg, L.max_parts);
    if (L.qout && L.no_gauss) {
        *nparts = 0;                 // the caller sketches q'_i later, together with another vector
        return 0;
    }
    if (L.qout) {
        switch (L.qtype) {
            case RGS_F64: launch_gauss_t<double>(ctx, sk->theta.as<double>(), sk->k, n, L.qout, L.ldq, 1, partials, gg, ctl); break;
            case RGS_F32: launch_gauss_t<float>(ctx, sk->theta.as<double>(), sk->k, n, L.qout, L.ldq, 1, partials, gg, ctl); break;
            default: launch_gauss_t<__nv_bfloat16>(ctx, sk->theta.as<double>(), sk->k, n, L.qout, L.ldq, 1, partials, gg, ctl); break;
        }
    } else {
        launch_gauss_t<double>(ctx, sk->theta.as<double>(), sk->k, n, L.w, L.ldw, L.wcols, partials, gg, ctl);
    }
    *nparts = gg;
    return gg;
}

int rgs_launch_gauss_sketch2(rgs_context* ctx, const rgs_sketch_obj* sk, int64_t n, const void* x1, int x1type,
                             const double* x2, double* part1, double* part2, const int* ctl) {
    const int gg = rgs_update_nparts(ctx, sk, n, 1);
    const double* th = sk->theta.as<double>();
    if (x1type == RGS_F64)
        gauss_sketch2_kernel<double><<<gg, 256, 0, ctx->stream>>>(th, sk->k, n, (const double*)x1, x2, part1, part2, ctl);
    else if (x1type == RGS_F32)
        gauss_sketch2_kernel<float><<<gg, 256, 0, ctx->stream>>>(th, sk->k, n, (const float*)x1, x2, part1, part2, ctl);
    else
        gauss_sketch2_kernel<__nv_bfloat16><<<gg, 256, 0, ctx->stream>>>(th, sk->k, n, (const __nv_bfloat16*)x1, x2,
                                                                        part1, part2, ctl);
    RGS_CUDA(cudaGetLastError());
    ctx->launches++;
    return gg;
}

void rgs_launch_reduce_partials(rgs_context* ctx, const double* partials, int nparts, int k, int ncols, double scale,
                                double* Y, int64_t ldy, bool df) {
    if (df)
        reduce_partials_kernel<true><<<dim3((k + 255) / 256, ncols), 256, 0, ctx->stream>>>(partials, nparts, k, scale, Y, ldy);
    else
        reduce_partials_kernel<false><<<dim3((k + 255) / 256, ncols), 256, 0, ctx->stream>>>(partials, nparts, k, scale, Y, ldy);
    RGS_CUDA(cudaGetLastError());
    ctx->launches++;
}

void rgs_launch_gaussian_theta(rgs_context* ctx, double* theta, int k, int64_t n, uint64_t seed) {
    const int64_t total = (int64_t)((k + 1) / 2) * n;
    const int64_t blocks = (total + 255) / 256;
    gaussian_theta_kernel<<<(unsigned)blocks, 256, 0, ctx->stream>>>(theta, k, n, (uint32_t)seed, (uint32_t)(seed >> 32));
    RGS_CUDA(cudaGetLastError());
}
