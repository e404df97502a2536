// The learned preconditioner: six 3x3 convolutions (2 -> 32 -> 32 -> 32 -> 32 -> 32 -> 1, ReLU
// between layers, zero padding) on H x W grids, with hand-written forward and backward kernels.
//
//  - conv3x3_tma_kernel: the convolution as an implicit GEMM (pixels x (tap, c_in) times
//    (tap, c_in) x c_out) on the tcgen05 tensor cores (BF16 operands from shared memory, FP32
//    accumulator in TMEM, one M = 128 pixels x N = c_out x K = 16 MMA per tap and channel step),
//    each 16 x 8 pixel tile's halo brought in by TMA tensor copies (one per 8-channel chunk, zeros
//    outside the grid); every tap's operand is a descriptor into the same halo.
//  - conv3x3_tc_kernel: the same with 8 x 16 pixel tiles whose halos are staged by per-thread
//    asynchronous copies (three column-shifted copies); used where no tensor map can be encoded.  The same kernel computes
//    the backward pass for the activations: the gradient of a layer's input is the convolution of
//    the output gradient with the taps flipped and c_in / c_out swapped, masked by ReLU'.
//  - dweight_mma_kernel: weight and bias gradients (sums over all pixels of the batch) as
//    GEMMs over the pixels on the tensor cores, FP32 accumulation.
//  - loss / Adam / packing kernels.
// Activations are BF16 in NHWC layout; FP32 master parameters are repacked into BF16 after
// every update.
#include "common.cuh"

#include <cuda.h>

#include <algorithm>
#include <cstdlib>
#include <cmath>
#include <new>
#include <vector>

using bf16 = __nv_bfloat16;
using namespace rgsdev;

namespace {

constexpr int NL = 6;
constexpr int C_IN[NL] = {2, 32, 32, 32, 32, 32};
constexpr int C_OUT[NL] = {32, 32, 32, 32, 32, 1};
constexpr int CS_IN[NL] = {16, 32, 32, 32, 32, 32};   // stored channels of each layer's input
constexpr int CO_P[NL] = {32, 32, 32, 32, 32, 8};     // output channels padded to n8 tiles
constexpr int TH = 8, TW = 16;                        // pixel tile of a CTA

constexpr int64_t layer_w_count(int l) { return (int64_t)C_OUT[l] * C_IN[l] * 9; }
constexpr int64_t layer_count(int l) { return layer_w_count(l) + C_OUT[l]; }
int64_t param_offset(int l) {
    int64_t o = 0;
    for (int i = 0; i < l; ++i) o += layer_count(i);
    return o;
}
int64_t total_params() { return param_offset(NL); }


__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

struct ConvArgs {
    const bf16* x;        // input, NHWC with CS channels
    const bf16* w;        // [9][CO][CS] (tap, output channel, input channel)
    const float* bias;    // [CO] (MODE 0, 1)
    void* out;            // MODE 0, 2: NHWC bf16 with CO channels; MODE 1: FP32 [b][y][x] (channel 0)
    const bf16* mask;     // MODE 2: NHWC bf16 with CO channels; output zeroed where mask <= 0
    const float* scale;   // MODE 1: optional per-sample factor
    int* status;          // the handle's status word: RGS_ERR_TIMEOUT if the tensor-core wait ran out
    int H, W;
};

// ------------------------------------------------------------------ tcgen05 building blocks
// Shared-memory matrix descriptor of a K-major operand without swizzle: core matrices of 8 rows x
// 16 bytes stored contiguously (128 bytes), LBO = byte distance between K-adjacent core matrices,
// SBO = between row-adjacent (8-row groups) ones; descriptor version 1 (bits 46-47).
__device__ __forceinline__ uint64_t tc_sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}
// Instruction descriptor of kind::f16: BF16 A and B (both K-major), FP32 accumulator, M x N.
__host__ __device__ constexpr uint32_t tc_idesc_bf16(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}
__device__ __forceinline__ void tc_mma(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(accumulate)
        : "memory");
}
// 32 (NC = 32) or 16 FP32 accumulator columns of TMEM lane (taddr's lane + thread's lane)
template <int NC>
__device__ __forceinline__ void tc_ld(uint32_t taddr, float (&v)[NC]) {
    uint32_t r[NC];
    if constexpr (NC == 32) {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
            "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
              "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
              "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
            : "r"(taddr));
    } else {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(taddr));
    }
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int c = 0; c < NC; ++c) v[c] = __uint_as_float(r[c]);
}

// Shared memory of conv3x3_tc_kernel: three copies of the input halo (columns shifted by dx = 0, 1,
// 2), the weights, the mbarrier and the TMEM address.
template <int CS, int NP>
struct ConvTcSmem {
    static constexpr int C8 = CS / 8;
    static constexpr int COPY = (TH + 2) * 2 * C8 * 128;        // bytes of one halo copy
    static constexpr int A_BYTES = 3 * COPY;                    // one tile's halo copies (two buffers)
    static constexpr int B_BYTES = 9 * (NP / 8) * C8 * 128;
    static constexpr int BYTES = 2 * A_BYTES + B_BYTES + 16;
};

// 16-byte asynchronous copy global -> shared; bytes = 0 writes zeros (the source is not read).
__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc, int bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(sdst)),
                 "l"(gsrc), "r"(bytes)
                 : "memory");
}

// MODE 0: bias + ReLU, BF16 out.  MODE 1: bias, FP32 channel 0 out (times scale).  MODE 2: ReLU'
// mask (backward for the activations), BF16 out.  The 3x3 convolution of 8 x 16 pixel tiles as
// an implicit GEMM on tcgen05: D (128 pixels x NP channels, FP32 in TMEM) = sum over the 9 taps
// and the CS / 16 channel steps of A_tap (pixels x 16 input channels) B_tap^T (NP output channels
// x 16 input channels), one M = 128, N = NP, K = 16 MMA each, issued by one thread.  A_tap is
// addressed inside a halo copy: copy dx stores the halo rows hy = 0..9 as two octets of 8 pixels
// (columns x0 - 1 + dx + 8 xo + 0..7) of 8-channel core matrices, so the pixels (y, x) of the
// tile at tap (dy, dx) are the octets (y + dy) * 2 + xo: an 8-row-group stride of C8 * 128 bytes
// from the start 2 dy C8 * 128.  NP: CO rounded up to 16 (zero weight rows).  The CTAs are
// persistent over tiles: the weights are staged once; the halo of a tile is staged by
// asynchronous copies (all of a thread's copies in flight at once) into one of two buffers while
// the tensor core works on the previous tile, whose MMAs commit to an mbarrier (one phase per
// tile) before the epilogue reads the accumulator from TMEM.
template <int CS, int CO, int MODE>
__global__ void __launch_bounds__(128) conv3x3_tc_kernel(ConvArgs a, int B) {
    constexpr int NP = CO < 16 ? 16 : CO;
    using SM = ConvTcSmem<CS, NP>;
    constexpr int C8 = SM::C8;
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* sB = smem + 2 * SM::A_BYTES;                        // halo buffers 0, 1 first
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + 2 * SM::A_BYTES + SM::B_BYTES);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tilesx = a.W / TW, tilesy = a.H / TH, ntiles = tilesx * tilesy * B;
    // the halo copies of tile t into buffer buf: chunk (dx, hy, xo, c8, px) = 8 channels of one
    // input pixel (zeros outside the grid), by asynchronous copies
    auto stage_halo = [&](int t, int buf) {
        const int b = t / (tilesx * tilesy), r = t % (tilesx * tilesy);
        const int y0 = (r / tilesx) * TH, x0 = (r % tilesx) * TW;
        const bf16* X = a.x + (size_t)b * a.H * a.W * CS;
        unsigned char* sA = smem + buf * SM::A_BYTES;
        for (int c = tid; c < 3 * (TH + 2) * 2 * C8 * 8; c += 128) {
            const int px = c & 7, c8 = (c >> 3) % C8, oct = (c >> 3) / C8;    // oct = (dx, hy, xo)
            const int xo = oct & 1, hy = (oct >> 1) % (TH + 2), dx = (oct >> 1) / (TH + 2);
            const int gy = y0 - 1 + hy, gx = x0 - 1 + dx + 8 * xo + px;
            const bool in = gy >= 0 && gy < a.H && gx >= 0 && gx < a.W;
            cp_async16(sA + dx * SM::COPY + ((hy * 2 + xo) * C8 + c8) * 128 + px * 16,
                       in ? X + ((size_t)gy * a.W + gx) * CS + c8 * 8 : X, in ? 16 : 0);
        }
    };
    // the weights, once: chunk (tap, n8, c8, row) = 8 input channels of output channel 8 n8 + row
    for (int c = tid; c < 9 * (NP / 8) * C8 * 8; c += 128) {
        const int row = c & 7, c8 = (c >> 3) % C8, tn = (c >> 3) / C8;      // tn = tap * (NP / 8) + n8
        const int n8 = tn % (NP / 8), tap = tn / (NP / 8);
        const int co = n8 * 8 + row;
        cp_async16(sB + ((tn * C8) + c8) * 128 + row * 16, co < CO ? a.w + ((size_t)tap * CO + co) * CS + c8 * 8 : a.w,
                   co < CO ? 16 : 0);
    }
    const uint32_t mbar_a = (uint32_t)__cvta_generic_to_shared(mbar);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar_a) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;"
                     ::"r"((uint32_t)__cvta_generic_to_shared(tslot)) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t taddr = *tslot;
    bool ok = true;
    uint32_t phase = 0;
    int buf = 0;
    if (blockIdx.x < ntiles) stage_halo(blockIdx.x, 0);
    for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, phase ^= 1u, buf ^= 1) {
        const int b = t / (tilesx * tilesy), r = t % (tilesx * tilesy);
        const int y0 = (r / tilesx) * TH, x0 = (r % tilesx) * TW;
        unsigned char* sA = smem + buf * SM::A_BYTES;
        asm volatile("cp.async.wait_all;" ::: "memory");        // the weights and tile t's halo
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // the operands, for the tensor core
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (tid == 0) {
            const uint32_t a0 = (uint32_t)__cvta_generic_to_shared(sA), b0 = (uint32_t)__cvta_generic_to_shared(sB);
            constexpr uint32_t idesc = tc_idesc_bf16(128, NP);
#pragma unroll 1
            for (int tap = 0; tap < 9; ++tap) {
                const int dy = tap / 3, dx = tap % 3;
#pragma unroll
                for (int kk = 0; kk < CS / 16; ++kk) {
                    const uint64_t ad = tc_sdesc(a0 + dx * SM::COPY + 2 * dy * C8 * 128 + kk * 256, 128, C8 * 128);
                    const uint64_t bd = tc_sdesc(b0 + tap * (NP / 8) * C8 * 128 + kk * 256, 128, C8 * 128);
                    tc_mma(taddr, ad, bd, idesc, (tap | kk) != 0 ? 1u : 0u);
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar_a)
                         : "memory");
        }
        // the next tile's halo into the other buffer, while the tensor core works on this one (that
        // buffer's last reader, the MMAs of the previous tile, completed in the previous iteration)
        if (t + (int)gridDim.x < ntiles) stage_halo(t + gridDim.x, buf ^ 1);
        // bounded wait for this tile's MMAs; a wait that runs out records RGS_ERR_TIMEOUT and ends
        // the CTA's tiles (decided for the whole CTA: every thread leaves the loop together)
        uint32_t seen = 0;
        for (int it = 0; it < (1 << 22) && !seen; ++it)
            asm volatile(
                "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                : "=r"(seen) : "r"(mbar_a), "r"(phase) : "memory");
        const bool done = __syncthreads_and((int)seen) != 0;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (!done) {
            if (tid == 0 && a.status) atomicCAS(a.status, 0, (int)RGS_ERR_TIMEOUT);
            ok = false;
        } else {
            float acc[NP];
            tc_ld<NP>(taddr + ((uint32_t)(warp * 32) << 16), acc);    // TMEM lanes 32 warp .. = pixels
            const int p = warp * 32 + lane, y = y0 + p / TW, x = x0 + p % TW;
            const size_t pix = ((size_t)b * a.H + y) * a.W + x;
            if constexpr (MODE == 1) {
                const float sc = a.scale ? a.scale[b] : 1.f;
                reinterpret_cast<float*>(a.out)[pix] = (acc[0] + a.bias[0]) * sc;
            } else {
                bf16* o = reinterpret_cast<bf16*>(a.out) + pix * CO;
#pragma unroll
                for (int c = 0; c < CO; c += 8) {
                    float v[8];
                    if constexpr (MODE == 0) {
#pragma unroll
                        for (int e = 0; e < 8; ++e) v[e] = fmaxf(acc[c + e] + a.bias[c + e], 0.f);
                    } else {
                        const uint4 mk = __ldg(reinterpret_cast<const uint4*>(a.mask + pix * CO + c));
                        const bf16* m = reinterpret_cast<const bf16*>(&mk);
#pragma unroll
                        for (int e = 0; e < 8; ++e) v[e] = __bfloat162float(m[e]) > 0.f ? acc[c + e] : 0.f;
                    }
                    uint4 pk;
                    __nv_bfloat162* q = reinterpret_cast<__nv_bfloat162*>(&pk);
#pragma unroll
                    for (int e = 0; e < 4; ++e) q[e] = __floats2bfloat162_rn(v[2 * e], v[2 * e + 1]);
                    *reinterpret_cast<uint4*>(o + c) = pk;
                }
            }
        }
        // TMEM is reused by the next tile only after every thread has read it
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;" ::"r"(taddr) : "memory");
}

// ---- the convolution with TMA-staged halos
// One 4-D tensor map per 8-channel chunk of the input (dims: 8 channels, W, H, B; strides 2 CS,
// 2 CS W, 2 CS W H bytes): a tile's halo chunk is one cp.async.bulk.tensor of a box of 8 channels
// x 10 columns x 18 rows, landing as rows of 16 bytes, pixel (h, w) at (10 h + w) * 16, with
// zeros where the box leaves the grid.  The tile is 16 rows x 8 columns, so the 8-row groups of
// the M = 128 pixels are 8 consecutive columns of one row: for tap (dy, dx) and channel step kk
// the operand A is the descriptor at (10 dy + dx) * 16 into chunks 2 kk, 2 kk + 1, with an 8-row
// group stride of 160 bytes and the chunk stride as K step (no shifted copies).  Thread 0 keeps
// CONV_STAGES tiles' halos in flight, issues a tile's MMAs into one of two TMEM accumulators and
// commits them to that accumulator's mbarrier; all threads read the other accumulator (the
// previous tile) meanwhile.  A stage is refilled once the MMAs that read it have completed.  Same
// MMAs in the same order as conv3x3_tc_kernel: bit-identical outputs.
constexpr int TH2 = 16, TW2 = 8;                               // pixel tile (rows x columns)
constexpr int HALO_H = TH2 + 2, HALO_W = TW2 + 2;
constexpr int CHUNK_BYTES = HALO_H * HALO_W * 16;              // one chunk's box
constexpr int CHUNK_STRIDE = (CHUNK_BYTES + 127) / 128 * 128;  // chunks 128-byte aligned
constexpr int CONV_STAGES = 4;

struct ConvMaps {
    CUtensorMap m[4];                  // chunks 0 .. CS / 8 - 1
};

template <int CS, int NP>
struct ConvTmaSmem {
    static constexpr int C8 = CS / 8;
    static constexpr int STAGE = C8 * CHUNK_STRIDE;
    static constexpr int B_BYTES = 9 * (NP / 8) * C8 * 128;
    static constexpr int BYTES = CONV_STAGES * STAGE + B_BYTES + 8 * (CONV_STAGES + 2) + 16;
};

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(mbar)
        : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_poll(uint32_t mbar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok) : "r"(mbar), "r"(parity) : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_wait_limited(uint32_t mbar, uint32_t parity) {
    for (int it = 0; it < (1 << 22); ++it)
        if (mbar_poll(mbar, parity)) return true;
    return false;
}

template <int CS, int CO, int MODE>
__global__ void __launch_bounds__(128) conv3x3_tma_kernel(const __grid_constant__ ConvMaps maps, ConvArgs a, int B) {
    constexpr int NP = CO < 16 ? 16 : CO;
    using SM = ConvTmaSmem<CS, NP>;
    constexpr int C8 = SM::C8, NS = CONV_STAGES;
    constexpr int TCOLS = 2 * NP < 32 ? 32 : 2 * NP;             // two accumulators of NP columns
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* sB = smem + NS * SM::STAGE;
    uint64_t* full = reinterpret_cast<uint64_t*>(sB + SM::B_BYTES);
    uint64_t* mdone = full + NS;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mdone + 2);
    int* abort_flag = reinterpret_cast<int*>(tslot + 1);       // a halo wait of thread 0 ran out
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tilesx = a.W / TW2, tilesy = (a.H + TH2 - 1) / TH2, ntiles = tilesx * tilesy * B;
    const int G = gridDim.x;
    const int nmine = (int)blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / G + 1 : 0;
    const uint32_t full0 = (uint32_t)__cvta_generic_to_shared(full);
    const uint32_t mdone0 = (uint32_t)__cvta_generic_to_shared(mdone);
    const uint32_t stage0 = (uint32_t)__cvta_generic_to_shared(smem);
    auto coords = [&](int j, int& b, int& y0, int& x0) {
        const int t = (int)blockIdx.x + j * G;
        b = t / (tilesx * tilesy);
        const int r = t % (tilesx * tilesy);
        y0 = (r / tilesx) * TH2;
        x0 = (r % tilesx) * TW2;
    };
    // thread 0's bookkeeping: tiles whose halo copies were issued / seen landed, MMAs issued
    int issued = 0, landed = 0, mmas = 0;
    auto issue = [&](int j) {
        if (j >= nmine) return;
        int b, y0, x0;
        coords(j, b, y0, x0);
        const int s = j % NS;
        mbar_arrive_expect_tx(full0 + 8 * s, (uint32_t)(C8 * CHUNK_BYTES));
#pragma unroll
        for (int c = 0; c < C8; ++c)
            tma_load_4d(stage0 + s * SM::STAGE + c * CHUNK_STRIDE, &maps.m[c], 0, x0 - 1, y0 - 1, b, full0 + 8 * s);
        issued = j + 1;
    };
    // the barriers, and the first halos in flight while the weights are staged and TMEM allocated
    if (tid == 0) {
        for (int q = 0; q < NS + 2; ++q)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(full0 + 8 * q) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *abort_flag = 0;
        for (int j = 0; j < NS; ++j) issue(j);
    }
    // the weights, once (as in conv3x3_tc_kernel)
    for (int c = tid; c < 9 * (NP / 8) * C8 * 8; c += 128) {
        const int row = c & 7, c8 = (c >> 3) % C8, tn = (c >> 3) / C8;
        const int n8 = tn % (NP / 8), tap = tn / (NP / 8);
        const int co = n8 * 8 + row;
        cp_async16(sB + ((tn * C8) + c8) * 128 + row * 16, co < CO ? a.w + ((size_t)tap * CO + co) * CS + c8 * 8 : a.w,
                   co < CO ? 16 : 0);
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     ::"r"((uint32_t)__cvta_generic_to_shared(tslot)), "n"(TCOLS) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");    // the weights, for the tensor core
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t taddr = *tslot;
    bool ok = true;
    for (int j = 0; j <= nmine && ok; ++j) {
        // tile j's MMAs into accumulator j % 2, once its halo has landed (thread 0)
        if (tid == 0 && j < nmine) {
            const int s = j % NS;
            if (!mbar_wait_limited(full0 + 8 * s, (uint32_t)((j / NS) & 1))) {
                *abort_flag = 1;
            } else {
                landed = j + 1;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t a0 = stage0 + s * SM::STAGE, b0 = (uint32_t)__cvta_generic_to_shared(sB);
                const uint32_t dcol = taddr + (uint32_t)((j & 1) * NP);
                constexpr uint32_t idesc = tc_idesc_bf16(128, NP);
#pragma unroll
                for (int tap = 0; tap < 9; ++tap) {
                    const int dy = tap / 3, dx = tap % 3;
#pragma unroll
                    for (int kk = 0; kk < CS / 16; ++kk) {
                        const uint64_t ad = tc_sdesc(a0 + 2 * kk * CHUNK_STRIDE + (dy * HALO_W + dx) * 16, CHUNK_STRIDE,
                                                     HALO_W * 16);
                        const uint64_t bd = tc_sdesc(b0 + tap * (NP / 8) * C8 * 128 + kk * 256, 128, C8 * 128);
                        tc_mma(dcol, ad, bd, idesc, (tap | kk) != 0 ? 1u : 0u);
                    }
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                             ::"r"(mdone0 + 8 * (j & 1)) : "memory");
                mmas = j + 1;
            }
        }
        // the epilogue of tile j - 1 (all threads) from accumulator (j - 1) % 2
        if (j >= 1) {
            const int jp = j - 1;
            const bool seen = mbar_wait_limited(mdone0 + 8 * (jp & 1), (uint32_t)((jp >> 1) & 1));
            const bool done = __syncthreads_and((int)seen) != 0;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            if (!done) {
                if (tid == 0 && a.status) atomicCAS(a.status, 0, (int)RGS_ERR_TIMEOUT);
                ok = false;
            } else {
                if (tid == 0) issue(jp + NS);            // its stage is free: the MMAs that read it are done
                int b, y0, x0;
                coords(jp, b, y0, x0);
                float acc[NP];
                tc_ld<NP>(taddr + (uint32_t)((jp & 1) * NP) + ((uint32_t)(warp * 32) << 16), acc);
                const int m = warp * 32 + lane, y = y0 + m / TW2, x = x0 + m % TW2;
                if (y < a.H) {
                    const size_t pix = ((size_t)b * a.H + y) * a.W + x;
                    if constexpr (MODE == 1) {
                        const float sc = a.scale ? a.scale[b] : 1.f;
                        reinterpret_cast<float*>(a.out)[pix] = (acc[0] + a.bias[0]) * sc;
                    } else {
                        bf16* o = reinterpret_cast<bf16*>(a.out) + pix * CO;
#pragma unroll
                        for (int c = 0; c < CO; c += 8) {
                            float v[8];
                            if constexpr (MODE == 0) {
#pragma unroll
                                for (int e = 0; e < 8; ++e) v[e] = fmaxf(acc[c + e] + a.bias[c + e], 0.f);
                            } else {
                                const uint4 mk = __ldg(reinterpret_cast<const uint4*>(a.mask + pix * CO + c));
                                const bf16* mm = reinterpret_cast<const bf16*>(&mk);
#pragma unroll
                                for (int e = 0; e < 8; ++e) v[e] = __bfloat162float(mm[e]) > 0.f ? acc[c + e] : 0.f;
                            }
                            uint4 pk;
                            __nv_bfloat162* q = reinterpret_cast<__nv_bfloat162*>(&pk);
#pragma unroll
                            for (int e = 0; e < 4; ++e) q[e] = __floats2bfloat162_rn(v[2 * e], v[2 * e + 1]);
                            *reinterpret_cast<uint4*>(o + c) = pk;
                        }
                    }
                }
            }
        }
        // accumulator (j - 1) % 2 takes tile j + 1's MMAs next: every thread has read it
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        if (__syncthreads_or(*abort_flag)) {
            if (tid == 0 && a.status) atomicCAS(a.status, 0, (int)RGS_ERR_TIMEOUT);
            ok = false;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    if (!ok && tid == 0) {                               // copies and MMAs in flight end before the CTA does
        for (int j = landed; j < issued; ++j) mbar_wait_limited(full0 + 8 * (j % NS), (uint32_t)((j / NS) & 1));
        if (mmas > 0) mbar_wait_limited(mdone0 + 8 * ((mmas - 1) & 1), (uint32_t)(((mmas - 1) >> 1) & 1));
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "n"(TCOLS) : "memory");
}

__device__ __forceinline__ void ldsm_x4_trans(uint32_t (&r)[4], const bf16* p) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a));
}

// Weight and bias gradients on the tensor cores: for tap t,
// dW_t[co][ci] = sum_p dA[p][co] h[p + off(t)][ci] is a GEMM with the pixels as the reduction
// dimension.  One warp per tap (9 warps); a CTA stages an 8 x 16 pixel tile of dA and the
// halo of h (channel strides padded by 8 elements: conflict-free 8 x 8 ldmatrix rows), reads
// both transposed with ldmatrix.trans (pixels become the k index of the fragments) and
// accumulates (CO_S / 16) x (CI_S / 8) m16n8 tiles per warp in FP32 over its grid-stride
// tiles.  CI_S / CO_S are the stored channel counts (16 or 32); only the layer's CIN x COUT
// entries are written.  Each CTA writes its partial sums; reduce_grad_kernel adds them.
constexpr int DWM_THREADS = 288;
template <int CI_S, int CO_S, int CIN, int COUT>
__global__ void __launch_bounds__(DWM_THREADS) dweight_mma_kernel(const bf16* __restrict__ h,
                                                                  const bf16* __restrict__ dA, int B, int H, int W,
                                                                  float* __restrict__ part) {
    constexpr int HSI = CI_S + 8, HSO = CO_S + 8, MT = CO_S / 16, NT = CI_S / 8;
    constexpr int NOUT = COUT * CIN * 9 + COUT;
    __shared__ __align__(16) bf16 sh[(TH + 2) * (TW + 2) * HSI];
    __shared__ __align__(16) bf16 sd[TH * TW * HSO];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tap = warp, dy = tap / 3, dx = tap % 3;
    const int i8 = lane & 7, mat = lane >> 3;
    float acc[MT][NT][4];
#pragma unroll
    for (int a = 0; a < MT; ++a)
#pragma unroll
        for (int b = 0; b < NT; ++b)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[a][b][e] = 0.f;
    float bacc = 0.f;
    const int tilesx = W / TW, tilesy = H / TH;
    const int ntiles = B * tilesx * tilesy;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int b = tile / (tilesx * tilesy), r = tile % (tilesx * tilesy);
        const int y0 = (r / tilesx) * TH, x0 = (r % tilesx) * TW;
        __syncthreads();
        for (int c = tid; c < (TH + 2) * (TW + 2) * (CI_S / 8); c += DWM_THREADS) {
            const int pix = c / (CI_S / 8), ch = (c % (CI_S / 8)) * 8;
            const int gy = y0 - 1 + pix / (TW + 2), gx = x0 - 1 + pix % (TW + 2);
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (gy >= 0 && gy < H && gx >= 0 && gx < W)
                v = *reinterpret_cast<const uint4*>(h + (((size_t)b * H + gy) * W + gx) * CI_S + ch);
            *reinterpret_cast<uint4*>(sh + pix * HSI + ch) = v;
        }
        for (int c = tid; c < TH * TW * (CO_S / 8); c += DWM_THREADS) {
            const int pix = c / (CO_S / 8), ch = (c % (CO_S / 8)) * 8;
            const int gy = y0 + pix / TW, gx = x0 + pix % TW;
            *reinterpret_cast<uint4*>(sd + pix * HSO + ch) =
                *reinterpret_cast<const uint4*>(dA + (((size_t)b * H + gy) * W + gx) * CO_S + ch);
        }
        __syncthreads();
        if (tid < COUT)
            for (int p = 0; p < TH * TW; ++p) bacc += __bfloat162float(sd[p * HSO + tid]);
#pragma unroll 2
        for (int ks = 0; ks < TH; ++ks) {               // k step = one pixel row of the tile (16 pixels)
            uint32_t a[MT][4];
#pragma unroll
            for (int mt = 0; mt < MT; ++mt)
                ldsm_x4_trans(a[mt], sd + (ks * TW + i8 + ((mat >> 1) ? 8 : 0)) * HSO + mt * 16 + ((mat & 1) ? 8 : 0));
            uint32_t bf[NT][2];
#pragma unroll
            for (int np = 0; np < NT / 2; ++np) {
                uint32_t q[4];
                const int hpos = (ks + dy) * (TW + 2) + i8 + ((mat & 1) ? 8 : 0) + dx;
                ldsm_x4_trans(q, sh + hpos * HSI + np * 16 + ((mat >> 1) ? 8 : 0));
                bf[2 * np][0] = q[0];
                bf[2 * np][1] = q[1];
                bf[2 * np + 1][0] = q[2];
                bf[2 * np + 1][1] = q[3];
            }
#pragma unroll
            for (int mt = 0; mt < MT; ++mt)
#pragma unroll
                for (int nt = 0; nt < NT; ++nt) mma_bf16(acc[mt][nt], a[mt], bf[nt][0], bf[nt][1]);
        }
    }
    float* out = part + (size_t)blockIdx.x * NOUT;
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
        for (int nt = 0; nt < NT; ++nt)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int co = mt * 16 + g + (e >= 2 ? 8 : 0), ci = nt * 8 + 2 * t + (e & 1);
                if (co < COUT && ci < CIN) out[co * (CIN * 9) + ci * 9 + tap] = acc[mt][nt][e];
            }
    if (tid < COUT) out[COUT * CIN * 9 + tid] = bacc;
}

// grad[o] = sum over CTAs of part[cta][o], summed in a fixed order: a CTA takes 32 consecutive
// outputs (one per lane); warp w adds the partials w, w + 8, ... and the 8 warp sums are added
// in warp order.
__global__ void reduce_grad_kernel(const float* __restrict__ part, int nparts, int nout, float* __restrict__ grad) {
    __shared__ double ws[8][33];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int o = blockIdx.x * 32 + lane;
    double s = 0.0;
    if (o < nout)
        for (int c = warp; c < nparts; c += 8) s += part[(size_t)c * nout + o];
    ws[warp][lane] = s;
    __syncthreads();
    if (warp == 0 && o < nout) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += ws[w][lane];
        grad[o] = (float)t;
    }
}


// in: batch x 2 x H x W FP32 (NCHW) -> NHWC BF16 with 16 channels (2 used)
__global__ void pack_input_kernel(const float* __restrict__ in, int B, int HW, bf16* __restrict__ x0) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)B * HW) return;
    const int64_t b = i / HW, p = i % HW;
    alignas(16) bf16 v[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) v[c] = __float2bfloat16_rn(0.f);
    v[0] = __float2bfloat16_rn(in[(b * 2) * HW + p]);
    v[1] = __float2bfloat16_rn(in[(b * 2 + 1) * HW + p]);
    uint4* dst = reinterpret_cast<uint4*>(x0 + i * 16);
    dst[0] = reinterpret_cast<uint4*>(v)[0];
    dst[1] = reinterpret_cast<uint4*>(v)[1];
}

// Preconditioner input: channel 0 = x / rms(x), channel 1 = log kappa (single grid)
template <typename TX>
__global__ void pack_precond_kernel(const TX* __restrict__ x, const float* __restrict__ nrm, const double* __restrict__ lk,
                                    int HW, bf16* __restrict__ x0) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= HW) return;
    float xv;
    if constexpr (sizeof(TX) == 2) xv = __bfloat162float(x[i]);
    else xv = (float)x[i];
    const float inv = nrm[0] > 0.f ? 1.f / nrm[0] : 0.f;
    alignas(16) bf16 v[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) v[c] = __float2bfloat16_rn(0.f);
    v[0] = __float2bfloat16_rn(xv * inv);
    v[1] = __float2bfloat16_rn((float)lk[i]);
    uint4* dst = reinterpret_cast<uint4*>(x0 + (size_t)i * 16);
    dst[0] = reinterpret_cast<uint4*>(v)[0];
    dst[1] = reinterpret_cast<uint4*>(v)[1];
}

template <typename TX>
__global__ void norm_kernel(const TX* __restrict__ x, int n, float* __restrict__ out) {
    __shared__ double sh[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double v;
        if constexpr (sizeof(TX) == 2) v = __bfloat162float(x[i]);
        else v = (double)x[i];
        s = fma(v, v, s);
    }
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = threadIdx.x < (int)(blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
        t = warp_sum(t);
        if (threadIdx.x == 0) out[0] = (float)sqrt(t / n);       // root mean square
    }
}

// Loss terms per sample: stats[b] = (sum (out - t)^2, sum t^2), one CTA per (sample, chunk)
__global__ void loss_stats_kernel(const float* __restrict__ out, const float* __restrict__ tgt, int HW, int chunks,
                                  double* __restrict__ part) {
    __shared__ double sh[2][8];
    const int b = blockIdx.y;
    const int per = (HW + chunks - 1) / chunks;
    const int p0 = blockIdx.x * per, p1 = min(HW, p0 + per);
    double e2 = 0.0, t2 = 0.0;
    for (int p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
        const double o = out[(size_t)b * HW + p], t = tgt[(size_t)b * HW + p];
        e2 += (o - t) * (o - t);
        t2 += t * t;
    }
    e2 = warp_sum(e2);
    t2 = warp_sum(t2);
    if ((threadIdx.x & 31) == 0) { sh[0][threadIdx.x >> 5] = e2; sh[1][threadIdx.x >> 5] = t2; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, c = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { a += sh[0][w]; c += sh[1][w]; }
        part[((size_t)b * chunks + blockIdx.x) * 2] = a;
        part[((size_t)b * chunks + blockIdx.x) * 2 + 1] = c;
    }
}

// loss = mean_b e2_b / t2_b ; per-sample gradient scale 2 / (t2_b B)
__global__ void loss_final_kernel(const double* __restrict__ part, int B, int chunks, double* __restrict__ loss,
                                  float* __restrict__ gscale) {
    if (threadIdx.x != 0) return;
    double L = 0.0;
    for (int b = 0; b < B; ++b) {
        double e2 = 0.0, t2 = 0.0;
        for (int c = 0; c < chunks; ++c) { e2 += part[((size_t)b * chunks + c) * 2]; t2 += part[((size_t)b * chunks + c) * 2 + 1]; }
        L += t2 > 0.0 ? e2 / t2 : 0.0;
        gscale[b] = t2 > 0.0 ? (float)(2.0 / (t2 * B)) : 0.f;
    }
    loss[0] = L / B;
}

// dA6 = (out - t) * gscale_b, NHWC BF16 with 16 channels (channel 0 used)
__global__ void dout_kernel(const float* __restrict__ out, const float* __restrict__ tgt, const float* __restrict__ gs,
                            int B, int HW, bf16* __restrict__ d6) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)B * HW) return;
    const int b = (int)(i / HW);
    alignas(16) bf16 v[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) v[c] = __float2bfloat16_rn(0.f);
    v[0] = __float2bfloat16_rn((out[i] - tgt[i]) * gs[b]);
    uint4* dst = reinterpret_cast<uint4*>(d6 + i * 16);
    dst[0] = reinterpret_cast<uint4*>(v)[0];
    dst[1] = reinterpret_cast<uint4*>(v)[1];
}

// Residual-norm loss: aout_b = A_b out_b for the 5-point operator of each sample, given as
// S[b][c][y][x] with c = 0 centre, 1 west (x - 1), 2 east (x + 1), 3 north (y - 1), 4 south (y + 1)
__global__ void stencil_apply_kernel(const float* __restrict__ out, const float* __restrict__ S, int B, int H, int W,
                                     float* __restrict__ aout) {
    const int HW = H * W;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)B * HW) return;
    const int64_t b = i / HW;
    const int p = (int)(i % HW), y = p / W, x = p % W;
    const float* s = S + b * 5 * HW;
    const float* o = out + b * HW;
    float v = s[p] * o[p];
    if (x > 0) v = fmaf(s[HW + p], o[p - 1], v);
    if (x < W - 1) v = fmaf(s[2 * HW + p], o[p + 1], v);
    if (y > 0) v = fmaf(s[3 * HW + p], o[p - W], v);
    if (y < H - 1) v = fmaf(s[4 * HW + p], o[p + W], v);
    aout[i] = v;
}

// dL/d out = A_b^T g_b with g_b = (aout_b - t_b) gscale_b; NHWC BF16 with 16 channels (channel 0).
// Row q of A reaches p through its east (q = p - 1), west (q = p + 1), south (q = p - W) and
// north (q = p + W) coefficient.
__global__ void stencil_dout_kernel(const float* __restrict__ aout, const float* __restrict__ tgt,
                                    const float* __restrict__ gs, const float* __restrict__ S, int B, int H, int W,
                                    bf16* __restrict__ d6) {
    const int HW = H * W;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)B * HW) return;
    const int64_t b = i / HW;
    const int p = (int)(i % HW), y = p / W, x = p % W;
    const float* s = S + b * 5 * HW;
    const float* a = aout + b * HW;
    const float* t = tgt + b * HW;
    const float sc = gs[b];
    auto g = [&](int q) { return (a[q] - t[q]) * sc; };
    float v = s[p] * g(p);
    if (x > 0) v = fmaf(s[2 * HW + p - 1], g(p - 1), v);
    if (x < W - 1) v = fmaf(s[HW + p + 1], g(p + 1), v);
    if (y > 0) v = fmaf(s[4 * HW + p - W], g(p - W), v);
    if (y < H - 1) v = fmaf(s[3 * HW + p + W], g(p + W), v);
    alignas(16) bf16 o16[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) o16[c] = __float2bfloat16_rn(0.f);
    o16[0] = __float2bfloat16_rn(v);
    uint4* dst = reinterpret_cast<uint4*>(d6 + i * 16);
    dst[0] = reinterpret_cast<uint4*>(o16)[0];
    dst[1] = reinterpret_cast<uint4*>(o16)[1];
}

// Adam on the FP32 master parameters
__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// FP32 master parameters -> BF16 forward ([tap][co][ci], padded) and backward ([8 - tap][ci][co])
// weights and padded FP32 biases, for one layer.
__global__ void repack_kernel(const float* __restrict__ p, int cin, int cout, int cs_in, int co_p, int cs_d,
                              bf16* __restrict__ wf, bf16* __restrict__ wb, float* __restrict__ bias) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    const int nw = cout * cin * 9;
    if (o < nw) {
        const int co = o / (cin * 9), rem = o % (cin * 9), ci = rem / 9, tap = rem % 9;
        const bf16 v = __float2bfloat16_rn(p[o]);
        wf[((size_t)tap * co_p + co) * cs_in + ci] = v;
        if (wb) wb[((size_t)(8 - tap) * 32 + ci) * cs_d + co] = v;
    } else if (o < nw + cout) {
        bias[o - nw] = p[o];
    }
}

// Fan-in uniform initialisation from Philox (stream 8): U(-b, b), b = 1 / sqrt(9 c_in); biases 0.
// Each layer shrinks the activations' variance (by about 6 with the ReLU), so the initial
// output is small and the residual-norm loss starts near 1 instead of at ||A out||^2 >> 1.
__global__ void init_kernel(float* __restrict__ p, int64_t off, int64_t nw, int64_t nb, int cin, uint32_t k0, uint32_t k1) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nw + nb) return;
    if (i >= nw) { p[off + i] = 0.f; return; }
    uint32_t c[4] = {(uint32_t)(off + i), 0u, 0u, 8u};
    philox4x32_10(c, k0, k1);
    const double u = u53(c[0], c[1]);
    const double bound = 1.0 / sqrt(9.0 * cin);
    p[off + i] = (float)((2.0 * u - 1.0) * bound);
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (null if unavailable)
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
    static const EncodeTiledFn fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return (EncodeTiledFn) nullptr;
        }
        return reinterpret_cast<EncodeTiledFn>(p);
    }();
    return fn;
}

// The input's chunk maps: chunk c = channels 8c .. 8c + 7 of the NHWC BF16 tensor x (CS channels)
bool encode_conv_maps(ConvMaps& m, const bf16* x, int CS, int W, int H, int B) {
    const EncodeTiledFn fn = encode_tiled();
    if (!fn) return false;
    for (int c = 0; c < CS / 8; ++c) {
        const cuuint64_t dims[4] = {8, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)B};
        const cuuint64_t strides[3] = {(cuuint64_t)CS * 2, (cuuint64_t)CS * 2 * W, (cuuint64_t)CS * 2 * W * H};
        const cuuint32_t box[4] = {8, HALO_W, HALO_H, 1};
        const cuuint32_t estr[4] = {1, 1, 1, 1};
        if (fn(&m.m[c], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<bf16*>(x + 8 * c), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return false;
    }
    return true;
}

template <int CS, int NT, int MODE>
void launch_conv(rgs_context* ctx, const ConvArgs& a0, int B) {
    constexpr int CO = NT * 8, NP = CO < 16 ? 16 : CO;
    constexpr int smem = ConvTcSmem<CS, NP>::BYTES;
    ConvArgs a = a0;
    a.status = ctx->ctl.as<int>() + kStatusWord;
    // TMA-staged halos when the tensor maps can be encoded (RGS_CONV_TMA=0 in the environment:
    // the halos staged by per-thread asynchronous copies)
    const char* tma_env = std::getenv("RGS_CONV_TMA");
    ConvMaps maps{};
    if (!(tma_env && tma_env[0] == '0') && encode_conv_maps(maps, a.x, CS, a.W, a.H, B)) {
        constexpr int tsmem = ConvTmaSmem<CS, NP>::BYTES;
        auto kern = conv3x3_tma_kernel<CS, CO, MODE>;
        RGS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, tsmem));
        RGS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
        // one wave: as many CTAs per SM as the shared memory holds (TMEM: 2 NP columns each)
        const int per_sm = std::max(1, std::min(8, (227 * 1024) / (tsmem + 1024)));
        const int ntiles = (a.W / TW2) * ((a.H + TH2 - 1) / TH2) * B;
        const int grid = std::max(1, std::min(ntiles, per_sm * ctx->num_sms));
        kern<<<grid, 128, tsmem, ctx->stream>>>(maps, a, B);
        RGS_CUDA(cudaGetLastError());
        ctx->launches++;
        return;
    }
    auto kern = conv3x3_tc_kernel<CS, CO, MODE>;
    RGS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    RGS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    // one wave of resident CTAs: as many per SM as the shared memory holds, at most 8 (8 x 32 TMEM
    // columns of the 512)
    const int per_sm = std::max(1, std::min(8, (227 * 1024) / (smem + 1024)));
    const int ntiles = (a.W / TW) * (a.H / TH) * B;
    const int grid = std::max(1, std::min(ntiles, per_sm * ctx->num_sms));
    kern<<<grid, 128, smem, ctx->stream>>>(a, B);
    RGS_CUDA(cudaGetLastError());
    ctx->launches++;
}

}  // namespace

struct rgs_convnet_obj {
    rgs_handle h = nullptr;
    int H = 0, W = 0, max_batch = 0;
    int64_t step = 0;
    DevBuf params, grad, adam_m, adam_v;     // FP32, total_params()
    DevBuf wf[NL], wb[NL], bias[NL];         // BF16 packed weights, FP32 padded biases
    DevBuf act[NL];                          // act[0]: packed input (16 ch); act[l]: output of layer l (32 ch)
    DevBuf out;                              // FP32 network output (max_batch x H x W)
    DevBuf aout;                             // FP32 A out (residual-norm loss)
    DevBuf dA[2], d6;                        // backward activation gradients (ping-pong) and dA_6
    DevBuf part;                             // per-CTA partial gradients
    DevBuf lpart, scal;                      // loss partials; scalars (loss, scales, norm)
};

namespace {

void repack_all(rgs_convnet_obj* net) {
    rgs_context* h = net->h;
    for (int l = 0; l < NL; ++l) {
        const int n = (int)layer_count(l);
        const int cs_d = (l == NL - 1) ? 16 : 32;     // channels of dA_l as stored
        repack_kernel<<<(n + 255) / 256, 256, 0, h->stream>>>(
            net->params.as<float>() + param_offset(l), C_IN[l], C_OUT[l], CS_IN[l], CO_P[l], cs_d,
            net->wf[l].as<bf16>(), l > 0 ? net->wb[l].as<bf16>() : nullptr, net->bias[l].as<float>());
        RGS_CUDA(cudaGetLastError());
    }
    h->launches += NL;
}

// Forward pass of `batch` grids whose packed input is act[0]; output FP32 into out (times scale).
void forward(rgs_convnet_obj* net, int batch, float* out, const float* scale) {
    rgs_context* h = net->h;
    for (int l = 0; l < NL; ++l) {
        ConvArgs a{};
        a.x = net->act[l].as<bf16>();
        a.w = net->wf[l].as<bf16>();
        a.bias = net->bias[l].as<float>();
        a.H = net->H;
        a.W = net->W;
        if (l == 0) {
            a.out = net->act[1].ptr;
            launch_conv<16, 4, 0>(h, a, batch);
        } else if (l < NL - 1) {
            a.out = net->act[l + 1].ptr;
            launch_conv<32, 4, 0>(h, a, batch);
        } else {
            a.out = out;
            a.scale = scale;
            launch_conv<32, 1, 1>(h, a, batch);
        }
    }
}

int dweight_grid(const rgs_context* h) { return 2 * h->num_sms; }

template <int CSH, int CIN, int CSD, int COUT>
void launch_dweight(rgs_convnet_obj* net, int l, const bf16* hprev, const bf16* dA, int B) {
    rgs_context* h = net->h;
    const int grid = dweight_grid(h);
    const int nout = COUT * CIN * 9 + COUT;
    dweight_mma_kernel<CSH, CSD, CIN, COUT><<<grid, DWM_THREADS, 0, h->stream>>>(hprev, dA, B, net->H, net->W,
                                                                                  net->part.as<float>());
    RGS_CUDA(cudaGetLastError());
    reduce_grad_kernel<<<(nout + 31) / 32, 256, 0, h->stream>>>(net->part.as<float>(), grid, nout,
                                                                net->grad.as<float>() + param_offset(l));
    RGS_CUDA(cudaGetLastError());
    h->launches += 2;
}

// loss, gradient into net->grad; returns device pointer to the loss
double* loss_and_backward(rgs_convnet_obj* net, int B, const float* target, const float* stencil) {
    rgs_context* h = net->h;
    const int HW = net->H * net->W;
    const int chunks = 16;
    double* loss = net->scal.as<double>();                  // scal: [0] loss, [1] norm, [2..] scales
    float* gscale = reinterpret_cast<float*>(loss + 2);
    const int64_t tot = (int64_t)B * HW;
    const unsigned eg = (unsigned)((tot + 255) / 256);
    const float* fit = net->out.as<float>();                // what is compared with the target
    if (stencil) {
        stencil_apply_kernel<<<eg, 256, 0, h->stream>>>(net->out.as<float>(), stencil, B, net->H, net->W,
                                                        net->aout.as<float>());
        RGS_CUDA(cudaGetLastError());
        fit = net->aout.as<float>();
        h->launches++;
    }
    loss_stats_kernel<<<dim3(chunks, B), 256, 0, h->stream>>>(fit, target, HW, chunks, net->lpart.as<double>());
    RGS_CUDA(cudaGetLastError());
    loss_final_kernel<<<1, 32, 0, h->stream>>>(net->lpart.as<double>(), B, chunks, loss, gscale);
    RGS_CUDA(cudaGetLastError());
    if (stencil)
        stencil_dout_kernel<<<eg, 256, 0, h->stream>>>(fit, target, gscale, stencil, B, net->H, net->W,
                                                       net->d6.as<bf16>());
    else
        dout_kernel<<<eg, 256, 0, h->stream>>>(fit, target, gscale, B, HW, net->d6.as<bf16>());
    RGS_CUDA(cudaGetLastError());
    h->launches += 3;
    // layer 6: dW from (h_5, dA_6); dA_5 = (conv^T dA_6) masked by h_5 > 0
    launch_dweight<32, 32, 16, 1>(net, 5, net->act[5].as<bf16>(), net->d6.as<bf16>(), B);
    {
        ConvArgs a{};
        a.x = net->d6.as<bf16>();
        a.w = net->wb[5].as<bf16>();
        a.out = net->dA[0].ptr;
        a.mask = net->act[5].as<bf16>();
        a.H = net->H;
        a.W = net->W;
        launch_conv<16, 4, 2>(h, a, B);
    }
    int cur = 0;
    for (int l = NL - 2; l >= 0; --l) {       // layers 5 .. 1 (0-based 4 .. 0)
        const bf16* dAl = net->dA[cur].as<bf16>();
        if (l == 0) {
            launch_dweight<16, 2, 32, 32>(net, 0, net->act[0].as<bf16>(), dAl, B);
        } else {
            launch_dweight<32, 32, 32, 32>(net, l, net->act[l].as<bf16>(), dAl, B);
            ConvArgs a{};
            a.x = dAl;
            a.w = net->wb[l].as<bf16>();
            a.out = net->dA[cur ^ 1].ptr;
            a.mask = net->act[l].as<bf16>();
            a.H = net->H;
            a.W = net->W;
            launch_conv<32, 4, 2>(h, a, B);
            cur ^= 1;
        }
    }
    return loss;
}

void pack_training_input(rgs_convnet_obj* net, int B, const float* in) {
    const int64_t tot = (int64_t)B * net->H * net->W;
    pack_input_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, net->h->stream>>>(in, B, net->H * net->W,
                                                                               net->act[0].as<bf16>());
    RGS_CUDA(cudaGetLastError());
    net->h->launches++;
}

// out[0:n] = r / rms(r), out[n:2n] = log kappa (FP32), with rms(r) = ||r|| / sqrt(n) summed in FP64
// by one CTA (the grids of the learned preconditioner are at most a few hundred thousand points).
__global__ void __launch_bounds__(1024) convnet_input_kernel(int64_t n, const double* __restrict__ r,
                                                             const double* __restrict__ lk, float* __restrict__ out) {
    __shared__ double sh[33];
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += 1024) s = fma(r[i], r[i], s);
    s = block_sum<1024>(s, sh);
    const double rms = sqrt(s / (double)n);
    const double inv = rms > 0.0 ? 1.0 / rms : 0.0;
    for (int64_t i = threadIdx.x; i < n; i += 1024) {
        out[i] = (float)(r[i] * inv);
        out[n + i] = (float)lk[i];
    }
}

// out[c][row] (5 x n FP32): the coefficients of each row of a 5-point operator on an H x W grid (x
// fastest) by offset, c = 0 centre, 1 west (-1), 2 east (+1), 3 north (-W), 4 south (+W); a thread
// per row sums its entries per channel (repeated entries add).  An entry at another offset sets
// *bad.
__global__ void csr_stencil_kernel(int64_t n, int W, const int32_t* __restrict__ rowptr,
                                   const int32_t* __restrict__ colind, const double* __restrict__ val,
                                   float* __restrict__ out, int* bad) {
    const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= n) return;
    double c[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int q = rowptr[row]; q < rowptr[row + 1]; ++q) {
        const int64_t d = (int64_t)colind[q] - row;
        const int ch = d == 0 ? 0 : d == -1 ? 1 : d == 1 ? 2 : d == -W ? 3 : d == W ? 4 : -1;
        if (ch < 0) {
            atomicExch(bad, 1);
            continue;
        }
        c[ch] += val[q];
    }
#pragma unroll
    for (int t = 0; t < 5; ++t) out[t * n + row] = (float)c[t];
}

template <class F>
rgs_status guarded(rgs_handle h, F&& f) {
    try {
        f();
        if (h) h->last_error.clear();
        return RGS_OK;
    } catch (const RgsError& e) {
        if (h) h->last_error = e.msg;
        return e.status;
    } catch (const std::bad_alloc&) {
        if (h) h->last_error = "host allocation failed";
        return RGS_ERR_ALLOC;
    } catch (...) {
        if (h) h->last_error = "unexpected exception";
        return RGS_ERR_INVALID_ARG;
    }
}

}  // namespace

int64_t rgs_convnet_grid_points(const void* netp) {
    const rgs_convnet_obj* net = static_cast<const rgs_convnet_obj*>(netp);
    return (int64_t)net->H * net->W;
}

// z = rms(x) net(x / rms(x), log kappa) on one grid (the flexible-GMRES preconditioner),
// rms(x) = ||x|| / sqrt(H W)
void rgs_convnet_apply_precond(rgs_context* ctx, void* netp, const double* logkappa, const void* x, int xtype,
                               float* z) {
    rgs_convnet_obj* net = static_cast<rgs_convnet_obj*>(netp);
    RGS_REQUIRE(net->h != nullptr, "network without handle");
    const int HW = net->H * net->W;
    float* nrm = reinterpret_cast<float*>(net->scal.as<double>() + 1);
    if (xtype == RGS_F64) {
        norm_kernel<double><<<1, 1024, 0, ctx->stream>>>((const double*)x, HW, nrm);
        pack_precond_kernel<double><<<(HW + 255) / 256, 256, 0, ctx->stream>>>((const double*)x, nrm, logkappa, HW,
                                                                                net->act[0].as<bf16>());
    } else if (xtype == RGS_F32) {
        norm_kernel<float><<<1, 1024, 0, ctx->stream>>>((const float*)x, HW, nrm);
        pack_precond_kernel<float><<<(HW + 255) / 256, 256, 0, ctx->stream>>>((const float*)x, nrm, logkappa, HW,
                                                                               net->act[0].as<bf16>());
    } else {
        norm_kernel<bf16><<<1, 1024, 0, ctx->stream>>>((const bf16*)x, HW, nrm);
        pack_precond_kernel<bf16><<<(HW + 255) / 256, 256, 0, ctx->stream>>>((const bf16*)x, nrm, logkappa, HW,
                                                                              net->act[0].as<bf16>());
    }
    RGS_CUDA(cudaGetLastError());
    ctx->launches += 2;
    cudaStream_t keep = net->h->stream;
    net->h->stream = ctx->stream;
    forward(net, 1, z, nrm);
    net->h->stream = keep;
}

extern "C" {

int64_t rgs_convnet_num_params(void) { return total_params(); }

rgs_status rgs_convnet_input(rgs_handle h, int64_t n, const double* r, const double* logkappa, float* out) {
    if (!h) return RGS_ERR_INVALID_ARG;
    return guarded(h, [&] {
        RGS_REQUIRE(n >= 1 && r && logkappa && out, "need n >= 1 and r, logkappa, out");
        RGS_REQUIRE(!rgs_is_host_pointer(r) && !rgs_is_host_pointer(logkappa) && !rgs_is_host_pointer(out),
                    "r, logkappa and out must be device pointers");
        convnet_input_kernel<<<1, 1024, 0, h->stream>>>(n, r, logkappa, out);
        RGS_CUDA(cudaGetLastError());
    });
}

rgs_status rgs_csr_to_stencil(rgs_handle h, const rgs_csr* A, int32_t H, int32_t W, float* out) {
    if (!h) return RGS_ERR_INVALID_ARG;
    return guarded(h, [&] {
        RGS_REQUIRE(A && A->rowptr && A->colind && A->val && out, "null CSR array or out");
        RGS_REQUIRE(H >= 1 && W >= 1 && A->n == (int64_t)H * W, "the operator's n differs from H x W");
        RGS_REQUIRE(!rgs_is_host_pointer(out), "out must be a device pointer");
        int* bad = h->ctl.as<int>() + kFlagWord;
        RGS_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), h->stream));
        csr_stencil_kernel<<<(unsigned)((A->n + 255) / 256), 256, 0, h->stream>>>(A->n, W, A->rowptr, A->colind, A->val,
                                                                                 out, bad);
        RGS_CUDA(cudaGetLastError());
        int hb = 0;
        RGS_CUDA(cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
        RGS_CUDA(cudaStreamSynchronize(h->stream));
        RGS_REQUIRE(hb == 0, "not a 5-point operator on this grid");
    });
}

rgs_status rgs_convnet_create(rgs_handle h, int32_t height, int32_t width, int32_t max_batch, uint64_t seed,
                              rgs_convnet* out) {
    if (!h || !out) return RGS_ERR_INVALID_ARG;
    *out = nullptr;
    rgs_convnet_obj* net = new (std::nothrow) rgs_convnet_obj();
    if (!net) return RGS_ERR_ALLOC;
    rgs_status st = guarded(h, [&] {
        RGS_REQUIRE(height >= TH && width >= TW && height % TH == 0 && width % TW == 0,
                    "grid must be a multiple of 8 x 16");
        RGS_REQUIRE(max_batch >= 1, "max_batch must be >= 1");
        net->h = h;
        net->H = height;
        net->W = width;
        net->max_batch = max_batch;
        const int64_t P = total_params();
        const size_t HW = (size_t)height * width;
        net->params.ensure(P * 4);
        net->grad.ensure(P * 4);
        net->adam_m.ensure(P * 4);
        net->adam_v.ensure(P * 4);
        RGS_CUDA(cudaMemsetAsync(net->adam_m.ptr, 0, P * 4, h->stream));
        RGS_CUDA(cudaMemsetAsync(net->adam_v.ptr, 0, P * 4, h->stream));
        for (int l = 0; l < NL; ++l) {
            net->wf[l].ensure(sizeof(bf16) * 9 * CO_P[l] * CS_IN[l]);
            RGS_CUDA(cudaMemsetAsync(net->wf[l].ptr, 0, net->wf[l].bytes, h->stream));
            if (l > 0) {
                const int cs_d = (l == NL - 1) ? 16 : 32;
                net->wb[l].ensure(sizeof(bf16) * 9 * 32 * cs_d);
                RGS_CUDA(cudaMemsetAsync(net->wb[l].ptr, 0, net->wb[l].bytes, h->stream));
            }
            net->bias[l].ensure(sizeof(float) * CO_P[l]);
            RGS_CUDA(cudaMemsetAsync(net->bias[l].ptr, 0, net->bias[l].bytes, h->stream));
            const int64_t nw = layer_w_count(l), nb = C_OUT[l];
            init_kernel<<<(unsigned)((nw + nb + 255) / 256), 256, 0, h->stream>>>(
                net->params.as<float>(), param_offset(l), nw, nb, C_IN[l], (uint32_t)seed, (uint32_t)(seed >> 32));
            RGS_CUDA(cudaGetLastError());
        }
        net->act[0].ensure(sizeof(bf16) * HW * 16 * max_batch);
        for (int l = 1; l < NL; ++l) net->act[l].ensure(sizeof(bf16) * HW * 32 * max_batch);
        net->out.ensure(sizeof(float) * HW * max_batch);
        net->aout.ensure(sizeof(float) * HW * max_batch);
        net->dA[0].ensure(sizeof(bf16) * HW * 32 * max_batch);
        net->dA[1].ensure(sizeof(bf16) * HW * 32 * max_batch);
        net->d6.ensure(sizeof(bf16) * HW * 16 * max_batch);
        net->part.ensure(sizeof(float) * (size_t)dweight_grid(h) * (32 * 32 * 9 + 32));
        net->lpart.ensure(sizeof(double) * 2 * 16 * (size_t)max_batch);
        net->scal.ensure(sizeof(double) * (4 + (size_t)max_batch));
        repack_all(net);
        RGS_CUDA(cudaStreamSynchronize(h->stream));
    });
    if (st != RGS_OK) {
        delete net;
        return st;
    }
    *out = net;
    return RGS_OK;
}

rgs_status rgs_convnet_destroy(rgs_convnet net) {
    if (!net) return RGS_ERR_INVALID_ARG;
    delete net;
    return RGS_OK;
}

rgs_status rgs_convnet_get_params(rgs_handle h, rgs_convnet net, float* host, int64_t count) {
    if (!h || !net || !host) return RGS_ERR_INVALID_ARG;
    return guarded(h, [&] {
        RGS_REQUIRE(count == total_params(), "count must equal rgs_convnet_num_params()");
        RGS_CUDA(cudaMemcpyAsync(host, net->params.ptr, count * 4, cudaMemcpyDeviceToHost, h->stream));
        RGS_CUDA(cudaStreamSynchronize(h->stream));
    });
}

rgs_status rgs_convnet_set_params(rgs_handle h, rgs_convnet net, const float* host, int64_t count) {
    if (!h || !net || !host) return RGS_ERR_INVALID_ARG;
    return guarded(h, [&] {
        RGS_REQUIRE(count == total_params(), "count must equal rgs_convnet_num_params()");
        RGS_CUDA(cudaMemcpyAsync(net->params.ptr, host, count * 4, cudaMemcpyHostToDevice, h->stream));
        repack_all(net);
        RGS_CUDA(cudaStreamSynchronize(h->stream));
    });
}

rgs_status rgs_convnet_forward(rgs_handle h, rgs_convnet net, int32_t batch, const float* in, float* out) {
    if (!h || !net || !in || !out) return RGS_ERR_INVALID_ARG;
    return guarded(h, [&] {
        RGS_REQUIRE(batch >= 1 && batch <= net->max_batch, "batch must be in [1, max_batch]");
        cudaStream_t keep = net->h->stream;
        net->h->stream = h->stream;
        pack_training_input(net, batch, in);
        forward(net, batch, out, nullptr);
        net->h->stream = keep;
    });
}

rgs_status rgs_convnet_loss_grad(rgs_handle h, rgs_convnet net, int32_t batch, const float* in, const float* target,
                                 const float* stencil, double* loss, float* grad_host) {
    if (!h || !net || !in || !target) return RGS_ERR_INVALID_ARG;
    return guarded(h, [&] {
        RGS_REQUIRE(batch >= 1 && batch <= net->max_batch, "batch must be in [1, max_batch]");
        cudaStream_t keep = net->h->stream;
        net->h->stream = h->stream;
        pack_training_input(net, batch, in);
        forward(net, batch, net->out.as<float>(), nullptr);
        double* dl = loss_and_backward(net, batch, target, stencil);
        net->h->stream = keep;
        if (loss) RGS_CUDA(cudaMemcpyAsync(loss, dl, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
        if (grad_host)
            RGS_CUDA(cudaMemcpyAsync(grad_host, net->grad.ptr, total_params() * 4, cudaMemcpyDeviceToHost, h->stream));
        RGS_CUDA(cudaStreamSynchronize(h->stream));
    });
}

rgs_status rgs_convnet_train_step(rgs_handle h, rgs_convnet net, int32_t batch, const float* in, const float* target,
                                  const float* stencil, float lr, double* loss) {
    if (!h || !net || !in || !target) return RGS_ERR_INVALID_ARG;
    return guarded(h, [&] {
        RGS_REQUIRE(batch >= 1 && batch <= net->max_batch, "batch must be in [1, max_batch]");
        cudaStream_t keep = net->h->stream;
        net->h->stream = h->stream;
        pack_training_input(net, batch, in);
        forward(net, batch, net->out.as<float>(), nullptr);
        double* dl = loss_and_backward(net, batch, target, stencil);
        net->step += 1;
        const float b1 = 0.9f, b2 = 0.999f;
        const float c1 = 1.f - std::pow(b1, (float)net->step), c2 = 1.f - std::pow(b2, (float)net->step);
        const int64_t P = total_params();
        adam_kernel<<<(unsigned)((P + 255) / 256), 256, 0, h->stream>>>(net->params.as<float>(), net->grad.as<float>(),
                                                                         net->adam_m.as<float>(), net->adam_v.as<float>(),
                                                                         P, lr, b1, b2, 1e-8f, c1, c2);
        RGS_CUDA(cudaGetLastError());
        h->launches++;
        repack_all(net);
        net->h->stream = keep;
        if (loss) {
            RGS_CUDA(cudaMemcpyAsync(loss, dl, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
            RGS_CUDA(cudaStreamSynchronize(h->stream));
        }
    });
}

}  // extern "C"
