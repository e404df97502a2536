// rgmres_solve_batched: many independent restarted RGMRES solves in one persistent launch.
//
// The cooperative grid is split into teams of CTAs; each team owns one instance (or, with
// more instances than CTAs, a list of instances solved one after the other) and runs the
// whole restarted RGS-Arnoldi / GMRES of Alg. 3 and Eq. hls for it with team-local barriers:
//
//   cycle:  R   r = b - A x (FP64), q'_0 = r, ||r||                       [all CTAs of the team]
//           for i = 0 .. m:
//             U   q'_i = sigma_{i-1} w - Q'_{0:i} coef  (i >= 1)              [all]
//             S   w = A q'_i and the sketches Theta q'_i, Theta w          [all, one pass over Theta]
//             L   r_ii, s_i, least squares for the next coefficients,
//                 Givens rotation of Hessenberg column i-1, stop test     [first CTA]
//           H   y from the rotated Hessenberg system                      [first CTA]
//           X   x += Q' (sigma .* y)                                      [all]
//
// The sketch is Gaussian: Theta_b = G[0:k_b, 0:n_b] / sqrt(k_b) with G one shared k_max x n_max
// matrix of N(0, 1) draws (Philox, the layout of the single-instance Gaussian sketch) rounded
// to bfloat16 -- any leading block of an i.i.d. Gaussian matrix is an i.i.d. Gaussian matrix,
// the rounded entries still form a sub-Gaussian embedding, and the 2-byte entries keep the
// whole of G resident in L2 while the teams stream their bases.  Products with it are
// accumulated in double-float (about 2^-48).  The kernel sketches with G itself: scaling Theta
// by a constant scales every sketch, r_ii, the Givens right-hand side and the inner threshold
// alike and leaves the normalised sketches, the Hessenberg matrix and the iterates unchanged,
// so the factor 1/sqrt(k_b) is never applied.  The least-squares problem of step 2 of Alg. 2 is
// solved through a QR factorisation of the sketched basis S built by classical Gram-Schmidt
// with reorthogonalisation (CGS2) in FP64 plus the explicit inverse of its triangular factor,
// which a single CTA applies as matrix-vector products.
#include "common.cuh"
#include "givens.cuh"

#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

using bf16 = __nv_bfloat16;
using namespace rgsdev;

namespace {

constexpr int BT = 256;                  // threads per CTA
constexpr int KB_MAX = 192;              // sketch rows of one instance
constexpr int MB_MAX = 127;              // restart length of one instance
constexpr int GROUPS = 4;                // row groups of the sketch accumulation
constexpr int GL = BT / GROUPS;          // threads per group; a thread owns sketch rows tl + GL j
constexpr int LPT = KB_MAX / GL;         // sketch rows per thread
// RR, the rows per thread of the streaming phases (and of the tensor-core sketch's tile of grid
// rows), is a template parameter: kernels for RR = 2 and RR = 4 are built and the autotuner
// chooses between them.

// Device-side description of one instance and its workspace.
struct BInst {
    int64_t n;
    const int32_t* rowptr;
    const int32_t* colind;
    const double* val;
    const double* b;
    double* x;
    int m, k, max_cycles, fixed;
    double rtol, inner;
    void* Q;             // n x (m+1) stored basis q' (F32 or F64), ld ldq
    int64_t ldq;
    double* w;           // n: A q'_i, and the residual at a restart
    double* part;        // team size x 2k partial sketches / partial sums
    double* U;           // k x (m+1): orthonormal basis of span(S) (CGS2), ld k
    double* RS;          // (m+1) x (m+1): triangular factor of S, column-major
    double* RSi;         // (m+1) x (m+1): its inverse
    double* R;           // (m+2) x (m+1): Arnoldi coefficients, column j = coefficients of A q_{j-1}
    double* sigma;       // m+1: 1 / r_ii
    double* coef;        // m+1: sigma_j c_j for the next update
    double* cs;          // m+1 Givens cosines
    double* sn;          // m+1 Givens sines
    double* g;           // m+2 rotated right-hand side
    double* Hr;          // (m+1) x (m+1) rotated Hessenberg factor, ld m+1
    double* y;           // m+1: sigma .* y
    double* scal;        // [0] ||b|| [1] ||Theta b|| [2] inner threshold [3] ||p_i|| [4] last rel
    int* flags;          // [0] stop step of the cycle (0: none) [1] continue the solve [2] steps
    unsigned* bar;       // team barrier word
    double* hist;        // max_cycles + 1 residuals (or null)
    int* out;            // [0] status [1] cycles [2] total steps [3] converged
};

struct BatchParams {
    const BInst* inst;
    const int* cta_team;     // team of each CTA (-1: idle)
    const int* cta_rank;     // rank of the CTA in its team
    const int* team_size;
    const int* team_begin;   // team t solves team_list[team_begin[t] .. team_begin[t+1])
    const int* team_list;
    const bf16* theta;       // shared G, column pairs interleaved: (l, c) at (c >> 1) * 2 ldt + 2 l + (c & 1)
    int ldt;                 // rows of G (k_max)
    int64_t nt;              // columns of G (n_max rounded up to even)
    int* ctl;                // [kStatusWord] first error, [kAbortWord] abort
};

__device__ __forceinline__ float2 split_df(double v) {
    const float h = __double2float_rn(v);
    return make_float2(h, __double2float_rn(v - (double)h));
}

// acc += t * (a.x + a.y), t a float (exact products via FMA, double-float sum)
__device__ __forceinline__ df df_fma(float t, float2 a, df acc) {
    const float ph = t * a.x;
    float pe = fmaf(t, a.x, -ph);
    pe = fmaf(t, a.y, pe);
    return df_add(acc, {ph, pe});
}

template <typename TQ> __device__ __forceinline__ double ldq(const TQ* p) { return (double)__ldcg(p); }
template <typename TQ> __device__ __forceinline__ TQ to_q(double v) { return (TQ)v; }

// Team barrier on one word (the grid barrier's sign-flip scheme on a team of T CTAs).
__device__ bool team_barrier(unsigned* word, int T, int rank, int* ctl) {
    __shared__ int ok_sh;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        if (T > 1) {
            const unsigned add = rank == 0 ? 0x80000000u - (unsigned)(T - 1) : 1u;
            const long long budget = wait_budget(ctl);
            const unsigned old = atom_add_acq_rel(word, add);
            const long long start = clock64();
            unsigned spins = 0;
            while (((old ^ ld_acquire(word)) & 0x80000000u) == 0u) {
                if (clock64() - start > budget) {
                    atomicCAS(ctl + kStatusWord, 0, (int)RGS_ERR_TIMEOUT);
                    atomicExch(ctl + kAbortWord, 1);
                    ok = 0;
                    break;
                }
                if ((++spins & 63u) == 0 && *reinterpret_cast<volatile int*>(ctl + kAbortWord) != 0) {
                    ok = 0;
                    break;
                }
            }
        } else {
            __threadfence();
            if (*reinterpret_cast<volatile int*>(ctl + kAbortWord) != 0) ok = 0;
        }
        ok_sh = ok;
    }
    __syncthreads();
    return ok_sh != 0;
}

__device__ __forceinline__ double cta_sum(double v, double* red) { return block_sum<BT>(v, red); }

// Partial sketches of the CTA's rows [r0, r1).  MODE 0: vector b.  MODE 1: q'_i and
// w = A q'_i (w stored).  MODE 2: q'_i.  Writes part[rank*2k + l] and part[rank*2k + k + l].
template <int RR>
struct SketchSmem {
    float2 sv0[BT], sv1[BT];                 // double-float split of the tile's vectors
    df red0[GROUPS][KB_MAX], red1[GROUPS][KB_MAX];
    __align__(16) bf16 pc[8][RR * BT + 8];   // tensor-core path: bf16 pieces of the two vectors
};

template <typename TQ, int MODE, int RR>
__device__ void sketch_phase(const BatchParams& P, const BInst& I, int i, int64_t r0, int64_t r1, int rank,
                             SketchSmem<RR>& S) {
    float2* sv0 = S.sv0;
    float2* sv1 = S.sv1;
    auto& red0 = S.red0;
    auto& red1 = S.red1;
    const int t = threadIdx.x, grp = t / GL, tl = t % GL, k = I.k;
    df acc0[LPT], acc1[LPT];
#pragma unroll
    for (int j = 0; j < LPT; ++j) acc0[j] = acc1[j] = {0.f, 0.f};
    const TQ* qcol = static_cast<const TQ*>(I.Q) + (size_t)i * I.ldq;
    for (int64_t c0 = r0; c0 < r1; c0 += BT) {
        const int64_t c = c0 + t;
        double v0 = 0.0, v1 = 0.0;
        if (c < r1) {
            if (MODE == 0) {
                v0 = I.b[c];
            } else {
                v0 = ldq(qcol + c);
                if (MODE == 1) {
                    double s = 0.0;
                    for (int q = I.rowptr[c]; q < I.rowptr[c + 1]; ++q) s = fma(I.val[q], ldq(qcol + I.colind[q]), s);
                    v1 = s;
                    I.w[c] = s;
                }
            }
        }
        sv0[t] = split_df(v0);
        sv1[t] = split_df(v1);
        __syncthreads();
        const int nt = (int)(r1 - c0 < (int64_t)BT ? r1 - c0 : (int64_t)BT);
        const int e = min(nt, grp * GL + GL);
        // the entries of G come from L2 or HBM: load those of RU rows before using any of them
        constexpr int RU = 8;
        for (int rb = grp * GL; rb < e; rb += RU) {
            float tv[RU][LPT];
#pragma unroll
            for (int u = 0; u < RU; ++u) {
                const int64_t cc = c0 + rb + u;
                const bf16* th = P.theta + (size_t)(cc >> 1) * 2 * P.ldt + (cc & 1);
#pragma unroll
                for (int j = 0; j < LPT; ++j) {
                    const int l = tl + j * GL;
                    tv[u][j] = (rb + u < e && l < k) ? __bfloat162float(th[2 * l]) : 0.f;
                }
            }
#pragma unroll
            for (int u = 0; u < RU; ++u) {
                if (rb + u < e) {
                    const float2 a0 = sv0[rb + u], a1 = sv1[rb + u];
#pragma unroll
                    for (int j = 0; j < LPT; ++j) {
                        acc0[j] = df_fma(tv[u][j], a0, acc0[j]);
                        if (MODE == 1) acc1[j] = df_fma(tv[u][j], a1, acc1[j]);
                    }
                }
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < LPT; ++j) {
        const int l = tl + j * GL;
        if (l < k) {
            red0[grp][l] = acc0[j];
            red1[grp][l] = acc1[j];
        }
    }
    __syncthreads();
    double* out = I.part + (size_t)rank * 2 * k;
    for (int l = t; l < k; l += BT) {
        df s0 = red0[0][l], s1 = red1[0][l];
        for (int q = 1; q < GROUPS; ++q) {
            s0 = df_add(s0, red0[q][l]);
            s1 = df_add(s1, red1[q][l]);
        }
        out[l] = (double)s0.h + (double)s0.l;
        if (MODE == 1) out[k + l] = (double)s1.h + (double)s1.l;
    }
}

__device__ __forceinline__ void mma_a02(float (&d)[4], uint32_t a0, uint32_t a2, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(0u), "r"(a2), "r"(0u), "r"(b0), "r"(b1));
}

// v = p0 + p1 + p2 with bfloat16 pieces (exact for an FP32 value, 24 significant bits otherwise)
__device__ __forceinline__ void split3(double v, bf16& p0, bf16& p1, bf16& p2) {
    p0 = __float2bfloat16_rn((float)v);
    const double r1 = v - (double)__bfloat162float(p0);
    p1 = __float2bfloat16_rn((float)r1);
    const double r2 = r1 - (double)__bfloat162float(p1);
    p2 = __float2bfloat16_rn((float)r2);
}

// The same partial sketches as sketch_phase, for FP32 bases on the tensor cores.  Each vector
// is split into three bfloat16 pieces (exact for FP32 values), so the 16 x 16 A operand of
// mma.m16n8k16 holds 6 piece rows (vector 0: rows 0-2, vector 1: rows 3-5) over 16 grid rows,
// and the B operand is a 16 x 8 block of G (grid rows x sketch rows), one 32-bit word per
// column pair of the interleaved layout.  Products are exact; the FP32 accumulator is flushed
// into double-float sums every 64 grid rows; the pieces are added at the end.
template <int MODE, int RR>
__device__ void sketch_phase_tc(const BatchParams& P, const BInst& I, int i, int64_t r0, int64_t r1, int rank,
                                SketchSmem<RR>& S) {
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31, g = lane >> 2, tq = lane & 3;
    const int k = I.k, ntiles = (k + 7) / 8;
    const float* qcol = static_cast<const float*>(I.Q) + (size_t)i * I.ldq;
    const uint32_t* G = reinterpret_cast<const uint32_t*>(P.theta);
    const int64_t npairs = P.nt / 2;
    constexpr int NJ = KB_MAX / 8 / (BT / 32);          // n-tiles per warp
    df sums[NJ][2];
    float acc[NJ][4];
#pragma unroll
    for (int j = 0; j < NJ; ++j) {
        sums[j][0] = sums[j][1] = {0.f, 0.f};
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[j][e] = 0.f;
    }
    for (int64_t c0 = r0; c0 < r1; c0 += RR * BT) {
        double v0[RR], v1[RR];
        int64_t cr[RR];
        int p0[RR], p1[RR];
#pragma unroll
        for (int q = 0; q < RR; ++q) {
            cr[q] = c0 + q * BT + t;
            v0[q] = v1[q] = 0.0;
            p0[q] = p1[q] = 0;
            if (cr[q] < r1) {
                if (MODE == 0) {
                    v0[q] = I.b[cr[q]];
                } else {
                    v0[q] = (double)__ldcg(qcol + cr[q]);
                    if (MODE == 1) {
                        p0[q] = I.rowptr[cr[q]];
                        p1[q] = I.rowptr[cr[q] + 1];
                    }
                }
            }
        }
        if (MODE == 1) {
            // w = A q'_i for the RR rows at once (independent loads), entries in CSR order
            int len = 0;
#pragma unroll
            for (int q = 0; q < RR; ++q) len = max(len, p1[q] - p0[q]);
            for (int e = 0; e < len; ++e)
#pragma unroll
                for (int q = 0; q < RR; ++q)
                    if (p0[q] + e < p1[q])
                        v1[q] = fma(I.val[p0[q] + e], (double)__ldcg(qcol + I.colind[p0[q] + e]), v1[q]);
#pragma unroll
            for (int q = 0; q < RR; ++q)
                if (cr[q] < r1) I.w[cr[q]] = v1[q];
        }
#pragma unroll
        for (int q = 0; q < RR; ++q) {
            split3(v0[q], S.pc[0][q * BT + t], S.pc[1][q * BT + t], S.pc[2][q * BT + t]);
            split3(v1[q], S.pc[3][q * BT + t], S.pc[4][q * BT + t], S.pc[5][q * BT + t]);
        }
        __syncthreads();
        const int nvalid = (int)(r1 - c0 < (int64_t)(RR * BT) ? r1 - c0 : (int64_t)(RR * BT));
        const int nks = (nvalid + 15) / 16;
        for (int k4 = 0; k4 < nks; k4 += 4) {
            uint32_t bw[4][NJ][2];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int64_t cp = (c0 + (int64_t)(k4 + u) * 16) / 2 + tq;
#pragma unroll
                for (int j = 0; j < NJ; ++j) {
                    const int l = (warp + 8 * j) * 8 + g;
                    const bool ok = k4 + u < nks && warp + 8 * j < ntiles && l < P.ldt;
                    bw[u][j][0] = (ok && cp < npairs) ? __ldg(G + (size_t)cp * P.ldt + l) : 0u;
                    bw[u][j][1] = (ok && cp + 4 < npairs) ? __ldg(G + (size_t)(cp + 4) * P.ldt + l) : 0u;
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (k4 + u < nks) {
                    const int kk = (k4 + u) * 16 + 2 * tq;
                    const uint32_t a0 = g < 6 ? *reinterpret_cast<const uint32_t*>(&S.pc[g][kk]) : 0u;
                    const uint32_t a2 = g < 6 ? *reinterpret_cast<const uint32_t*>(&S.pc[g][kk + 8]) : 0u;
#pragma unroll
                    for (int j = 0; j < NJ; ++j)
                        if (warp + 8 * j < ntiles) mma_a02(acc[j], a0, a2, bw[u][j][0], bw[u][j][1]);
                }
            }
#pragma unroll
            for (int j = 0; j < NJ; ++j) {
                sums[j][0] = df_add(sums[j][0], {acc[j][0], 0.f});
                sums[j][1] = df_add(sums[j][1], {acc[j][1], 0.f});
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[j][e] = 0.f;
            }
        }
        __syncthreads();
    }
    // add the three pieces of each vector: lanes 4g + tq with g = 0, 1, 2 (vector 0) and 3, 4, 5 (vector 1)
    double* out = I.part + (size_t)rank * 2 * k;
#pragma unroll
    for (int j = 0; j < NJ; ++j)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            df v = sums[j][e];
            const df v1 = {__shfl_down_sync(0xffffffffu, v.h, 4), __shfl_down_sync(0xffffffffu, v.l, 4)};
            const df v2 = {__shfl_down_sync(0xffffffffu, v.h, 8), __shfl_down_sync(0xffffffffu, v.l, 8)};
            v = df_add(df_add(v, v1), v2);
            const int l = (warp + 8 * j) * 8 + 2 * tq + e;
            if (warp + 8 * j < ntiles && l < k) {
                if (g == 0) out[l] = (double)v.h + (double)v.l;
                if (MODE == 1 && g == 3) out[k + l] = (double)v.h + (double)v.l;
            }
        }
}

template <typename TQ, int MODE, int RR>
__device__ __forceinline__ void sketch_any(const BatchParams& P, const BInst& I, int i, int64_t r0, int64_t r1,
                                           int rank, SketchSmem<RR>& S) {
    if constexpr (sizeof(TQ) == 4) sketch_phase_tc<MODE, RR>(P, I, i, r0, r1, rank, S);
    else sketch_phase<TQ, MODE, RR>(P, I, i, r0, r1, rank, S);
}

// The first CTA: sum of the team's partial vectors into dst (length len, offset off).
__device__ void reduce_parts(const BInst& I, int T, int off, int len, double* dst) {
    const int k2 = 2 * I.k;
    for (int l = threadIdx.x; l < len; l += BT) {
        double s = 0.0;
        for (int r = 0; r < T; ++r) s += __ldcg(I.part + (size_t)r * k2 + off + l);
        dst[l] = s;
    }
    __syncthreads();
}

// h[j] = U(:, j)^T v for j < ncol (one warp per column, in turn)
__device__ void cta_dots(const double* U, int k, int ncol, const double* v, double* h) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int j = warp; j < ncol; j += BT / 32) {
        double s = 0.0;
        for (int l = lane; l < k; l += 32) s = fma(U[(size_t)j * k + l], v[l], s);
        s = warp_sum(s);
        if (lane == 0) h[j] = s;
    }
    __syncthreads();
}

// v -= U(:, 0:ncol) h (thread per entry, four interleaved sums)
__device__ void cta_axpy(const double* U, int k, int ncol, const double* h, double* v) {
    for (int l = threadIdx.x; l < k; l += BT) {
        double a[4] = {0.0, 0.0, 0.0, 0.0};
        int j = 0;
        for (; j + 4 <= ncol; j += 4) {
#pragma unroll
            for (int q = 0; q < 4; ++q) a[q] = fma(U[(size_t)(j + q) * k + l], h[j + q], a[q]);
        }
        for (; j < ncol; ++j) a[0] = fma(U[(size_t)j * k + l], h[j], a[0]);
        v[l] -= (a[0] + a[1]) + (a[2] + a[3]);
    }
    __syncthreads();
}

// One least-squares / Givens step of the first CTA (see the file comment).  ss: s'_i, pp:
// Theta A q'_i (valid when i < m).  Returns false on a device error.
__device__ bool leader_step(const BInst& I, int i, double stop_tol, double* ss, double* pp, double* h1,
                            double* h2, double* red) {
    const int k = I.k, m = I.m, ld = m + 1;
    const int t = threadIdx.x;
    __shared__ int sh_stop, sh_bad;
    // the step's scalars (square roots, reciprocals) come from thread 0 through shared memory:
    // FP64 square roots and divisions are long sequences on this GPU's FP64 pipe
    __shared__ double sh_sc[4];
    double a = 0.0;
    for (int l = t; l < k; l += BT) a = fma(ss[l], ss[l], a);
    const double sum_s = cta_sum(a, red);
    if (t == 0) {
        const double r0 = sqrt(sum_s);
        sh_sc[0] = r0;
        sh_sc[1] = r0 > 0.0 ? 1.0 / r0 : 0.0;
        sh_stop = 0;
        sh_bad = !isfinite(r0) ? 1 : 0;
        // r_ii at the rounding level of ||p_i||: the Krylov space is invariant (happy breakdown)
        if (i > 0 && !(r0 > 16.0 * 0x1p-53 * __ldcg(I.scal + 3))) sh_stop = i;
        if (i == 0 && !(r0 > 0.0)) sh_bad = 1;
    }
    __syncthreads();
    if (sh_bad) return false;
    const double rii = sh_sc[0], sig = sh_sc[1];
    if (t == 0) I.sigma[i] = sig;
    // Givens rotation of Hessenberg column i-1 = [R(0:i-1, i); r_ii]
    if (i == 0) {
        if (t == 0) I.g[0] = rii;
    } else if (t < 32) {
        const double* Rc = I.R + (size_t)i * (m + 2);
        auto hcol = [&](int q) { return q < i ? Rc[q] : rii; };
        const double res = givens_column_warp(i - 1, hcol, I.cs, I.sn, I.g, I.Hr, ld);
        if (t == 0 && res <= stop_tol && sh_stop == 0) sh_stop = i;
    }
    __syncthreads();
    const bool more = sh_stop == 0 && i < m;
    if (more) {
        // append s_i = s'_i / r_ii to the QR factorisation of S by CGS2
        for (int l = t; l < k; l += BT) ss[l] *= sig;
        __syncthreads();
        double* Ui = I.U + (size_t)i * k;
        if (i > 0) {
            cta_dots(I.U, k, i, ss, h1);
            cta_axpy(I.U, k, i, h1, ss);
            cta_dots(I.U, k, i, ss, h2);
            cta_axpy(I.U, k, i, h2, ss);
        }
        a = 0.0;
        for (int l = t; l < k; l += BT) a = fma(ss[l], ss[l], a);
        const double sum_r = cta_sum(a, red);
        if (t == 0) {
            const double r0 = sqrt(sum_r);
            sh_sc[2] = r0;
            sh_sc[3] = 1.0 / r0;
        }
        __syncthreads();
        const double rho = sh_sc[2], irho = sh_sc[3];
        if (!(rho > 0.0) || !isfinite(rho)) return false;
        for (int l = t; l < k; l += BT) Ui[l] = ss[l] * irho;
        // R_S(0:i, i) and the new column of its inverse: Rinv(0:i-1, i) = -Rinv(0:i-1, 0:i-1) R_S(0:i-1, i) / rho
        double* RSc = I.RS + (size_t)i * ld;
        double* RIc = I.RSi + (size_t)i * ld;
        for (int q = t; q < i; q += BT) RSc[q] = h1[q] + h2[q];
        if (t == 0) RSc[i] = rho;
        __syncthreads();
        {   // one warp per entry, lanes along the row
            const int warp = t >> 5, lane = t & 31;
            for (int q = warp; q < i; q += BT / 32) {
                double s = 0.0;
                for (int j = q + lane; j < i; j += 32) s = fma(I.RSi[(size_t)j * ld + q], RSc[j], s);
                s = warp_sum(s);
                if (lane == 0) RIc[q] = -s * irho;
            }
        }
        if (t == 0) RIc[i] = irho;
        __syncthreads();
        // next coefficients: c = argmin ||S_{0:i} c - p_{i+1}||, p_{i+1} = sigma_i Theta A q'_i
        for (int l = t; l < k; l += BT) pp[l] *= sig;
        __syncthreads();
        a = 0.0;
        for (int l = t; l < k; l += BT) a = fma(pp[l], pp[l], a);
        const double sum_p = cta_sum(a, red);
        cta_dots(I.U, k, i + 1, pp, h1);
        double* Rn = I.R + (size_t)(i + 1) * (m + 2);
        {
            const int warp = t >> 5, lane = t & 31;
            for (int q = warp; q <= i; q += BT / 32) {
                double s = 0.0;
                for (int j = q + lane; j <= i; j += 32) s = fma(I.RSi[(size_t)j * ld + q], h1[j], s);
                s = warp_sum(s);
                if (lane == 0) {
                    Rn[q] = s;
                    I.coef[q] = s * I.sigma[q];
                }
            }
        }
        if (t == 0) I.scal[3] = sqrt(sum_p);
    }
    __syncthreads();
    if (t == 0) {
        if (sh_stop) I.flags[0] = sh_stop;
        __threadfence();
    }
    __syncthreads();
    return true;
}

// y = Hr(0:j, 0:j)^{-1} g(0:j), stored as sigma .* y (one warp); the reciprocals of the diagonal
// are formed by the lanes in parallel first, so the back substitution has no division in its chain
__device__ void hess_solve_warp(const BInst& I, int j, double* gs, double* dinv) {
    const int lane = threadIdx.x;
    const int ld = I.m + 1;
    for (int q = lane; q < j; q += 32) {
        gs[q] = I.g[q];
        dinv[q] = 1.0 / I.Hr[(size_t)q * ld + q];
    }
    __syncwarp();
    for (int r = j - 1; r >= 0; --r) {
        const double yr = gs[r] * dinv[r];
        for (int q = lane; q < r; q += 32) gs[q] = fma(-I.Hr[(size_t)r * ld + q], yr, gs[q]);
        if (lane == 0) I.y[r] = yr * I.sigma[r];
        __syncwarp();
    }
}

// q'_i = sg w - Q'_{0:i} cy over rows [r0, r1): RR rows per thread, the loads of 8 columns
// issued before their products; each row's FMA chain runs over j = 0 .. i-1 in order.
template <typename TQ, int RR>
__device__ void update_rows(TQ* Q, int64_t ldq, const double* w, double sg, const double* cy, int i, int64_t r0,
                            int64_t r1) {
    using A = TQ;
    for (int64_t base = r0 + threadIdx.x; base < r1; base += (int64_t)BT * RR) {
        A acc[RR];
        int64_t c[RR];
        bool ok[RR];
#pragma unroll
        for (int q = 0; q < RR; ++q) {
            c[q] = base + (int64_t)q * BT;
            ok[q] = c[q] < r1;
            if constexpr (sizeof(TQ) == 4) acc[q] = ok[q] ? __double2float_rn(sg * w[c[q]]) : 0.f;
            else acc[q] = ok[q] ? sg * w[c[q]] : 0.0;
        }
        int j = 0;
        for (; j + 8 <= i; j += 8) {
            A v[RR][8];
#pragma unroll
            for (int q = 0; q < RR; ++q)
#pragma unroll
                for (int u = 0; u < 8; ++u) v[q][u] = ok[q] ? Q[c[q] + (size_t)(j + u) * ldq] : (A)0;
#pragma unroll
            for (int u = 0; u < 8; ++u)
#pragma unroll
                for (int q = 0; q < RR; ++q) acc[q] = fma(-(A)cy[j + u], v[q][u], acc[q]);
        }
        for (; j < i; ++j)
#pragma unroll
            for (int q = 0; q < RR; ++q)
                if (ok[q]) acc[q] = fma(-(A)cy[j], Q[c[q] + (size_t)j * ldq], acc[q]);
#pragma unroll
        for (int q = 0; q < RR; ++q)
            if (ok[q]) Q[c[q] + (size_t)i * ldq] = acc[q];
    }
}

// x += Q'_{0:steps} cy (FP64 sums, columns in order), RR rows per thread
template <typename TQ, int RR>
__device__ void solution_rows(const TQ* Q, int64_t ld, const double* cy, int steps, double* x, int64_t r0,
                              int64_t r1) {
    for (int64_t base = r0 + threadIdx.x; base < r1; base += (int64_t)BT * RR) {
        double acc[RR];
        int64_t c[RR];
        bool ok[RR];
#pragma unroll
        for (int q = 0; q < RR; ++q) {
            c[q] = base + (int64_t)q * BT;
            ok[q] = c[q] < r1;
            acc[q] = 0.0;
        }
        int j = 0;
        for (; j + 8 <= steps; j += 8) {
            double v[RR][8];
#pragma unroll
            for (int q = 0; q < RR; ++q)
#pragma unroll
                for (int u = 0; u < 8; ++u) v[q][u] = ok[q] ? ldq(Q + c[q] + (size_t)(j + u) * ld) : 0.0;
#pragma unroll
            for (int u = 0; u < 8; ++u)
#pragma unroll
                for (int q = 0; q < RR; ++q) acc[q] = fma(v[q][u], cy[j + u], acc[q]);
        }
        for (; j < steps; ++j)
#pragma unroll
            for (int q = 0; q < RR; ++q)
                if (ok[q]) acc[q] = fma(ldq(Q + c[q] + (size_t)j * ld), cy[j], acc[q]);
#pragma unroll
        for (int q = 0; q < RR; ++q)
            if (ok[q]) x[c[q]] += acc[q];
    }
}

// r = b - A x over rows [r0, r1), stored as q'_0 (TQ); returns the thread's sum of r^2
template <typename TQ, int RR>
__device__ double residual_rows(const BInst& I, TQ* Q, int64_t r0, int64_t r1) {
    double a = 0.0;
    for (int64_t base = r0 + threadIdx.x; base < r1; base += (int64_t)BT * RR) {
        double s[RR];
        int64_t c[RR];
        int p0[RR], p1[RR];
#pragma unroll
        for (int q = 0; q < RR; ++q) {
            c[q] = base + (int64_t)q * BT;
            s[q] = 0.0;
            p0[q] = p1[q] = 0;
            if (c[q] < r1) {
                s[q] = I.b[c[q]];
                p0[q] = I.rowptr[c[q]];
                p1[q] = I.rowptr[c[q] + 1];
            }
        }
        int len = 0;
#pragma unroll
        for (int q = 0; q < RR; ++q) len = max(len, p1[q] - p0[q]);
        for (int e = 0; e < len; ++e)
#pragma unroll
            for (int q = 0; q < RR; ++q)
                if (p0[q] + e < p1[q]) s[q] = fma(-I.val[p0[q] + e], __ldcg(I.x + I.colind[p0[q] + e]), s[q]);
#pragma unroll
        for (int q = 0; q < RR; ++q)
            if (c[q] < r1) {
                Q[c[q]] = to_q<TQ>(s[q]);
                a = fma(s[q], s[q], a);
            }
    }
    return a;
}

template <typename TQ, int RR>
__device__ bool solve_one(const BatchParams& P, const BInst& I, int rank, int T) {
    __shared__ double red[BT / 32 + 1];
    __shared__ double ss[KB_MAX], pp[KB_MAX], h1[MB_MAX + 1], h2[MB_MAX + 1];
    __shared__ double cy[MB_MAX + 1];
    __shared__ int sh_flag[2];
    __shared__ SketchSmem<RR> sks;
    const int k = I.k, m = I.m, t = threadIdx.x;
    const bool leader = rank == 0;
    const int64_t chunk = ((I.n + T - 1) / T + 31) & ~(int64_t)31;
    const int64_t r0 = min(I.n, (int64_t)rank * chunk), r1 = min(I.n, r0 + chunk);
    TQ* Q = static_cast<TQ*>(I.Q);
    int* ctl = P.ctl;
    // ||b|| and ||Theta b||
    {
        double a = 0.0;
        for (int64_t c = r0 + t; c < r1; c += BT) a = fma(I.b[c], I.b[c], a);
        a = cta_sum(a, red);
        sketch_any<TQ, 0, RR>(P, I, 0, r0, r1, rank, sks);
        if (t == 0) I.part[(size_t)rank * 2 * k + k] = a;
        if (!team_barrier(I.bar, T, rank, ctl)) return false;
        if (leader) {
            reduce_parts(I, T, 0, k, ss);
            double q = 0.0;
            for (int l = t; l < k; l += BT) q = fma(ss[l], ss[l], q);
            const double sb = sqrt(cta_sum(q, red));
            if (t == 0) {
                double bb = 0.0;
                for (int r = 0; r < T; ++r) bb += __ldcg(I.part + (size_t)r * 2 * k + k);
                I.scal[0] = sqrt(bb);
                I.scal[1] = sb;
                I.scal[2] = I.fixed ? -1.0 : I.inner * I.rtol * sb;
                I.out[0] = I.out[1] = I.out[2] = I.out[3] = 0;
                I.flags[2] = 0;
                if (!(sqrt(bb) > 0.0) || !isfinite(bb)) I.out[0] = RGS_ERR_INVALID_ARG;
            }
        }
        if (!team_barrier(I.bar, T, rank, ctl)) return false;
        if (__ldcg(I.out) != 0) return true;
    }
    for (int cycle = 0;; ++cycle) {
        // R: r = b - A x, q'_0 = r, ||r||^2
        double a = residual_rows<TQ, RR>(I, Q, r0, r1);
        a = cta_sum(a, red);
        if (t == 0) I.part[(size_t)rank * 2 * k + k] = a;
        if (!team_barrier(I.bar, T, rank, ctl)) return false;
        if (leader && t == 0) {
            double rr = 0.0;
            for (int r = 0; r < T; ++r) rr += __ldcg(I.part + (size_t)r * 2 * k + k);
            const double rel = sqrt(rr) / I.scal[0];
            if (I.hist) I.hist[cycle] = rel;
            int go = 1;
            if (!isfinite(rel)) {
                I.out[0] = RGS_ERR_NONFINITE;
                go = 0;
            } else if (rel <= I.rtol) {
                I.out[3] = 1;
                go = 0;
            } else if (cycle >= I.max_cycles) {
                go = 0;
            }
            // a cycle that stopped on the inner test but missed rtol tightens the test
            if (go && cycle > 0 && I.scal[2] > 0.0 && I.flags[2] < m)
                I.scal[2] *= fmin(1.0, I.inner * I.rtol / rel);
            I.scal[4] = rel;
            I.out[1] = cycle;
            I.flags[1] = go;
            I.flags[0] = 0;
            __threadfence();
        }
        if (!team_barrier(I.bar, T, rank, ctl)) return false;
        if (t == 0) sh_flag[0] = __ldcg(I.flags + 1);
        __syncthreads();
        if (!sh_flag[0]) break;
        const double stop_tol = __ldcg(I.scal + 2);
        int steps = m;
        for (int i = 0; i <= m; ++i) {
            if (i > 0) {
                // U: q'_i = sigma_{i-1} w - Q'_{0:i} coef
                const double sg = __ldcg(I.sigma + i - 1);
                for (int j = t; j < i; j += BT) cy[j] = __ldcg(I.coef + j);
                __syncthreads();
                update_rows<TQ, RR>(Q, I.ldq, I.w, sg, cy, i, r0, r1);
                if (!team_barrier(I.bar, T, rank, ctl)) return false;
            }
            // S: w = A q'_i with the sketches of q'_i and w
            if (i < m) sketch_any<TQ, 1, RR>(P, I, i, r0, r1, rank, sks);
            else sketch_any<TQ, 2, RR>(P, I, i, r0, r1, rank, sks);
            if (!team_barrier(I.bar, T, rank, ctl)) return false;
            if (leader) {
                reduce_parts(I, T, 0, k, ss);
                if (i < m) reduce_parts(I, T, k, k, pp);
                if (!leader_step(I, i, stop_tol, ss, pp, h1, h2, red)) {
                    if (t == 0) {
                        atomicCAS(ctl + kStatusWord, 0, (int)RGS_ERR_NONFINITE);
                        I.out[0] = RGS_ERR_NONFINITE;
                        atomicExch(ctl + kAbortWord, 1);
                    }
                    return false;
                }
            }
            if (!team_barrier(I.bar, T, rank, ctl)) return false;
            if (t == 0) sh_flag[1] = __ldcg(I.flags + 0);
            __syncthreads();
            if (sh_flag[1] != 0) {
                steps = sh_flag[1];
                break;
            }
        }
        // H: y; X: x += Q' (sigma .* y)
        if (leader && t < 32) {
            hess_solve_warp(I, steps, h1, h2);
            if (t == 0) {
                I.flags[2] = steps;
                I.out[2] += steps;
                __threadfence();
            }
        }
        if (!team_barrier(I.bar, T, rank, ctl)) return false;
        for (int j = t; j < steps; j += BT) cy[j] = __ldcg(I.y + j);
        __syncthreads();
        solution_rows<TQ, RR>(Q, I.ldq, cy, steps, I.x, r0, r1);
        if (!team_barrier(I.bar, T, rank, ctl)) return false;
    }
    return true;
}

template <typename TQ, int RR>
__global__ void __launch_bounds__(BT) rgmres_batched_kernel(BatchParams P) {
    const int team = P.cta_team[blockIdx.x];
    if (team < 0) return;
    const int rank = P.cta_rank[blockIdx.x], T = P.team_size[team];
    for (int li = P.team_begin[team]; li < P.team_begin[team + 1]; ++li) {
        if (!solve_one<TQ, RR>(P, P.inst[P.team_list[li]], rank, T)) return;
    }
}

// Shared Gaussian G (k x n): entry (l, c) from counter (c, l >> 1, 0, 0), Box-Muller, rounded to
// bfloat16 (the single-instance Gaussian sketch before its 1/sqrt(k) scale).  Columns are stored
// in interleaved pairs, (l, c) at (c >> 1) * 2k + 2l + (c & 1), so that (l, c) and (l, c + 1)
// form one 32-bit word: the k-pair of a tensor-core fragment.
__global__ void batched_theta_kernel(bf16* G, int k, int64_t n, uint32_t key0, uint32_t key1) {
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
    bf16* col = G + (size_t)(c >> 1) * 2 * k + (c & 1);
    col[2 * (2 * pr)] = __float2bfloat16_rn(__double2float_rn(rad * cs));
    if (2 * pr + 1 < k) col[2 * (2 * pr + 1)] = __float2bfloat16_rn(__double2float_rn(rad * sn));
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

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

using BatchedKernel = void (*)(BatchParams);

// The kernel for a basis type and a rows-per-thread choice (2 or 4; anything else means 4).
BatchedKernel batched_kernel_for(int qtype, int rr) {
    if (qtype == RGS_F64) return rr == 2 ? rgmres_batched_kernel<double, 2> : rgmres_batched_kernel<double, 4>;
    return rr == 2 ? rgmres_batched_kernel<float, 2> : rgmres_batched_kernel<float, 4>;
}

}  // namespace

// Resident CTAs per SM of the batched kernel for a basis type and rows per thread (the
// cooperative grid's limit; at most 4).
int rgs_batched_max_blocks_per_sm(int qtype, int rr) {
    int per_sm = 0;
    RGS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batched_kernel_for(qtype, rr), BT, 0));
    return std::min(per_sm, 4);
}

extern "C" rgs_status rgmres_solve_batched(rgs_handle h, int32_t nbatch, const rgs_csr* A, const double* const* b,
                                           double* const* x, const rgmres_batch_opts* opts, uint64_t sketch_seed,
                                           rgmres_info* info) {
    if (!h) return RGS_ERR_INVALID_ARG;
    return guarded(h, [&] {
        RGS_REQUIRE(nbatch >= 0, "nbatch must be >= 0");
        if (nbatch == 0) return;
        RGS_REQUIRE(A && b && x && opts, "null array argument");
        const int qtype = opts[0].qtype;
        RGS_REQUIRE(qtype == RGS_F64 || qtype == RGS_F32, "batched solves store the basis in FP64 or FP32");
        int64_t nmax = 0;
        int kmax = 0;
        for (int i = 0; i < nbatch; ++i) {
            const rgmres_batch_opts& o = opts[i];
            RGS_REQUIRE(o.qtype == qtype, "every instance needs the same qtype");
            RGS_REQUIRE(o.restart >= 1 && o.restart <= MB_MAX, "restart must be in [1, 127]");
            RGS_REQUIRE(o.k >= o.restart + 1 && o.k <= KB_MAX, "need restart + 1 <= k <= 192");
            RGS_REQUIRE(o.max_cycles >= 0 && o.rtol >= 0.0 && o.inner_factor > 0.0, "bad max_cycles, rtol or inner_factor");
            RGS_REQUIRE(A[i].n >= 1 && A[i].rowptr && A[i].colind && A[i].val, "bad CSR");
            RGS_REQUIRE(b[i] && x[i], "null b or x");
            nmax = std::max(nmax, A[i].n);
            kmax = std::max(kmax, o.k);
        }
        // shared G (cached on the handle)
        rgs_context* ctx = h;
        const int64_t ncols = (nmax + 1) & ~(int64_t)1;
        const size_t gbytes = sizeof(bf16) * (size_t)kmax * ncols;
        if (ctx->batch_theta_seed != sketch_seed || ctx->batch_theta_k != kmax || ctx->batch_theta_n < ncols) {
            ctx->batch_theta.ensure(gbytes);
            RGS_CUDA(cudaMemsetAsync(ctx->batch_theta.ptr, 0, gbytes, ctx->stream));
            const int64_t tot = (int64_t)((kmax + 1) / 2) * nmax;
            batched_theta_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, ctx->stream>>>(
                ctx->batch_theta.as<bf16>(), kmax, nmax, (uint32_t)sketch_seed, (uint32_t)(sketch_seed >> 32));
            RGS_CUDA(cudaGetLastError());
            ctx->batch_theta_seed = sketch_seed;
            ctx->batch_theta_k = kmax;
            ctx->batch_theta_n = ncols;
        }
        // grid and teams: every CTA resident (cooperative launch)
        const BatchedKernel kern = batched_kernel_for(qtype, ctx->batch_rr);
        int per_sm = 0;
        RGS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BT, 0));
        RGS_REQUIRE(per_sm >= 1, "batched kernel does not fit on an SM");
        per_sm = std::min(per_sm, ctx->batch_blocks_per_sm > 0 ? ctx->batch_blocks_per_sm : 4);
        const int G = per_sm * ctx->num_sms;
        std::vector<double> work(nbatch);
        for (int i = 0; i < nbatch; ++i) work[i] = (double)A[i].n * (opts[i].k + opts[i].restart);
        std::vector<int> order(nbatch);
        std::iota(order.begin(), order.end(), 0);
        std::sort(order.begin(), order.end(), [&](int a, int c) { return work[a] > work[c]; });
        std::vector<int> team_size, team_begin, team_list;
        if (nbatch <= G) {
            // one instance per team: every team starts with one CTA and each spare CTA goes to
            // the team with the most work per CTA (balances the longest team's time)
            std::vector<int> ts(nbatch, 1);
            for (int left = G - nbatch; left > 0; --left) {
                int best = 0;
                for (int i = 1; i < nbatch; ++i)
                    if (work[i] / ts[i] > work[best] / ts[best]) best = i;
                if (work[best] / ts[best] < ctx->batch_min_team_work) break;    // not worth a barrier
                ts[best] += 1;
            }
            for (int i = 0; i < nbatch; ++i) {
                team_begin.push_back(i);
                team_list.push_back(i);
                team_size.push_back(ts[i]);
            }
            team_begin.push_back(nbatch);
        } else {
            // one CTA per team; instances dealt to the least-loaded team (longest first)
            std::vector<std::vector<int>> lists(G);
            std::vector<double> load(G, 0.0);
            for (int i : order) {
                const int tm = (int)(std::min_element(load.begin(), load.end()) - load.begin());
                lists[tm].push_back(i);
                load[tm] += work[i];
            }
            for (int tm = 0; tm < G; ++tm) {
                team_begin.push_back((int)team_list.size());
                for (int i : lists[tm]) team_list.push_back(i);
                team_size.push_back(1);
            }
            team_begin.push_back((int)team_list.size());
        }
        const int nteams = (int)team_size.size();
        std::vector<int> cta_team(G, -1), cta_rank(G, 0);
        {
            int c = 0;
            for (int tm = 0; tm < nteams; ++tm)
                for (int r = 0; r < team_size[tm]; ++r, ++c) {
                    cta_team[c] = tm;
                    cta_rank[c] = r;
                }
        }
        // workspace
        const size_t qsize = qtype == RGS_F64 ? 8 : 4;
        std::vector<size_t> off(nbatch + 1, 0);
        std::vector<int> tsz_of(nbatch, 1);
        for (int tm = 0; tm < nteams; ++tm)
            for (int q = team_begin[tm]; q < team_begin[tm + 1]; ++q) tsz_of[team_list[q]] = team_size[tm];
        auto inst_bytes = [&](int i) {
            const int64_t n = A[i].n;
            const int m = opts[i].restart, k = opts[i].k, ld = m + 1;
            const int64_t ldq = (n + 31) & ~(int64_t)31;
            size_t s = 0;
            s += align_up(qsize * (size_t)ldq * (m + 1), 256);            // Q
            s += align_up(8 * (size_t)n, 256);                              // w
            s += align_up(8 * (size_t)tsz_of[i] * 2 * k, 256);              // part
            s += align_up(8 * (size_t)k * (m + 1), 256);                    // U
            s += 2 * align_up(8 * (size_t)ld * ld, 256);                    // RS, RSi
            s += align_up(8 * (size_t)(m + 2) * (m + 1), 256);              // R
            s += 4 * align_up(8 * (size_t)(m + 2), 256);                    // sigma, coef, cs, sn
            s += align_up(8 * (size_t)(m + 2), 256);                        // g
            s += align_up(8 * (size_t)ld * ld, 256);                        // Hr
            s += align_up(8 * (size_t)(m + 2), 256);                        // y
            s += align_up(8 * 8, 256);                                      // scal
            s += align_up(4 * 8, 256);                                      // flags
            s += 256;                                                       // barrier word
            s += align_up(8 * (size_t)(opts[i].max_cycles + 1), 256);       // hist
            s += align_up(4 * 8, 256);                                      // out
            return s;
        };
        for (int i = 0; i < nbatch; ++i) off[i + 1] = off[i] + inst_bytes(i);
        ctx->batch_ws.ensure(off[nbatch]);
        RGS_CUDA(cudaMemsetAsync(ctx->batch_ws.ptr, 0, off[nbatch], ctx->stream));
        std::vector<BInst> hi(nbatch);
        char* base = ctx->batch_ws.as<char>();
        for (int i = 0; i < nbatch; ++i) {
            const rgmres_batch_opts& o = opts[i];
            const int64_t n = A[i].n;
            const int m = o.restart, k = o.k, ld = m + 1;
            char* p = base + off[i];
            auto take = [&](size_t bytes) {
                char* r = p;
                p += align_up(bytes, 256);
                return r;
            };
            BInst& I = hi[i];
            I.n = n;
            I.rowptr = A[i].rowptr;
            I.colind = A[i].colind;
            I.val = A[i].val;
            I.b = b[i];
            I.x = x[i];
            I.m = m;
            I.k = k;
            I.max_cycles = o.max_cycles;
            I.fixed = o.fixed_steps;
            I.rtol = o.rtol;
            I.inner = o.inner_factor;
            I.ldq = (n + 31) & ~(int64_t)31;
            I.Q = take(qsize * (size_t)I.ldq * (m + 1));
            I.w = (double*)take(8 * (size_t)n);
            I.part = (double*)take(8 * (size_t)tsz_of[i] * 2 * k);
            I.U = (double*)take(8 * (size_t)k * (m + 1));
            I.RS = (double*)take(8 * (size_t)ld * ld);
            I.RSi = (double*)take(8 * (size_t)ld * ld);
            I.R = (double*)take(8 * (size_t)(m + 2) * (m + 1));
            I.sigma = (double*)take(8 * (size_t)(m + 2));
            I.coef = (double*)take(8 * (size_t)(m + 2));
            I.cs = (double*)take(8 * (size_t)(m + 2));
            I.sn = (double*)take(8 * (size_t)(m + 2));
            I.g = (double*)take(8 * (size_t)(m + 2));
            I.Hr = (double*)take(8 * (size_t)ld * ld);
            I.y = (double*)take(8 * (size_t)(m + 2));
            I.scal = (double*)take(8 * 8);
            I.flags = (int*)take(4 * 8);
            I.bar = (unsigned*)take(256);
            I.hist = (double*)take(8 * (size_t)(o.max_cycles + 1));
            I.out = (int*)take(4 * 8);
        }
        // tables
        std::vector<int> tables;
        auto put = [&](const std::vector<int>& v) {
            const size_t o = tables.size();
            tables.insert(tables.end(), v.begin(), v.end());
            return o;
        };
        const size_t o_team = put(cta_team), o_rank = put(cta_rank), o_size = put(team_size),
                     o_begin = put(team_begin), o_list = put(team_list);
        ctx->batch_desc.ensure(sizeof(BInst) * nbatch + sizeof(int) * tables.size() + 256);
        BInst* d_inst = ctx->batch_desc.as<BInst>();
        int* d_tab = reinterpret_cast<int*>(ctx->batch_desc.as<char>() + align_up(sizeof(BInst) * nbatch, 256));
        RGS_CUDA(cudaMemcpyAsync(d_inst, hi.data(), sizeof(BInst) * nbatch, cudaMemcpyHostToDevice, ctx->stream));
        RGS_CUDA(cudaMemcpyAsync(d_tab, tables.data(), sizeof(int) * tables.size(), cudaMemcpyHostToDevice, ctx->stream));
        RGS_CUDA(cudaMemsetAsync(ctx->ctl.ptr, 0, kCtlWords * sizeof(int), ctx->stream));
        BatchParams P{};
        P.inst = d_inst;
        P.cta_team = d_tab + o_team;
        P.cta_rank = d_tab + o_rank;
        P.team_size = d_tab + o_size;
        P.team_begin = d_tab + o_begin;
        P.team_list = d_tab + o_list;
        P.theta = ctx->batch_theta.as<bf16>();
        P.ldt = kmax;
        P.nt = ctx->batch_theta_n;
        P.ctl = ctx->ctl.as<int>();
        void* args[] = {&P};
        // one persistent launch, issued through a CUDA graph: captured on the handle's private
        // stream (the bound stream may be the legacy default stream, which cannot capture) and
        // launched on the bound stream
        if (!ctx->capture_stream) RGS_CUDA(cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking));
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        RGS_CUDA(cudaStreamBeginCapture(ctx->capture_stream, cudaStreamCaptureModeThreadLocal));
        cudaLaunchAttribute attr{};
        attr.id = cudaLaunchAttributeCooperative;
        attr.val.cooperative = 1;
        cudaLaunchConfig_t cfg{};
        cfg.gridDim = dim3(G);
        cfg.blockDim = dim3(BT);
        cfg.dynamicSmemBytes = 0;
        cfg.stream = ctx->capture_stream;
        cfg.attrs = &attr;
        cfg.numAttrs = 1;
        const cudaError_t le = cudaLaunchKernelExC(&cfg, (const void*)kern, args);
        const cudaError_t ce = cudaStreamEndCapture(ctx->capture_stream, &graph);
        RGS_CUDA(le);
        RGS_CUDA(ce);
        cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
        if (ie == cudaSuccess) ie = cudaGraphLaunch(exec, ctx->stream);
        if (exec) cudaGraphExecDestroy(exec);
        cudaGraphDestroy(graph);
        RGS_CUDA(ie);
        ctx->launches = 1;
        // results
        std::vector<int> outs(8 * (size_t)nbatch);
        std::vector<double> sc(8 * (size_t)nbatch);
        for (int i = 0; i < nbatch; ++i) {
            RGS_CUDA(cudaMemcpyAsync(&outs[8 * (size_t)i], hi[i].out, 4 * 4, cudaMemcpyDeviceToHost, ctx->stream));
            RGS_CUDA(cudaMemcpyAsync(&sc[8 * (size_t)i], hi[i].scal, 8 * 5, cudaMemcpyDeviceToHost, ctx->stream));
            if (info && info[i].history)
                RGS_CUDA(cudaMemcpyAsync(info[i].history, hi[i].hist, 8 * (size_t)(opts[i].max_cycles + 1),
                                         cudaMemcpyDeviceToHost, ctx->stream));
        }
        int ctlv[kCtlWords];
        RGS_CUDA(cudaMemcpyAsync(ctlv, ctx->ctl.ptr, sizeof(ctlv), cudaMemcpyDeviceToHost, ctx->stream));
        RGS_CUDA(cudaStreamSynchronize(ctx->stream));
        if (info) {
            for (int i = 0; i < nbatch; ++i) {
                info[i].status = outs[8 * (size_t)i] != 0 ? outs[8 * (size_t)i]
                                                          : (outs[8 * (size_t)i + 3] ? RGS_OK : RGS_ERR_NOT_CONVERGED);
                info[i].cycles = outs[8 * (size_t)i + 1];
                info[i].total_steps = outs[8 * (size_t)i + 2];
                info[i].converged = outs[8 * (size_t)i + 3];
                info[i].rel_residual = sc[8 * (size_t)i + 4];
                info[i].fallback_cycle = -1;
                info[i].sell = 0;
                info[i].sketch_refreshes = 0;
            }
        }
        if (ctlv[kStatusWord] != 0)
            throw RgsError{(rgs_status)ctlv[kStatusWord], "device status in the batched solve"};
    });
}
