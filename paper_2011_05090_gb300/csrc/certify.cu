// A posteriori certificate of the epsilon-embedding property of Theta (Sec. 3.2, Prop. cert01).
//
// With V^Theta = Theta V, V^Phi = Phi V (Phi a second sketch, independent of V and Theta) and X
// such that V^Phi X is orthonormal, the singular values s of V^Theta X give
//     omega_bar = max(1 - (1 - eps*) s_min^2, (1 + eps*) s_max^2 - 1).
// GPU route, all FP64: the Gram matrices G_Phi = (V^Phi)^T V^Phi and G_Theta = (V^Theta)^T V^Theta
// (m x m); the Cholesky factor L of G_Phi (X = L^{-T}); C = L^{-1} G_Theta L^{-T}, whose
// eigenvalues are the s^2; Lanczos on C with two-pass classical Gram-Schmidt reorthogonalisation
// against the whole basis for m steps (the tridiagonal T_m is then similar to C up to rounding);
// the extreme eigenvalues of T_m by multisection with Sturm counts.  For the bases RGS produces,
// cond(G_Phi) = cond(V^Phi)^2 stays small (cond(S) is about 1-3), so forming the Gram matrices
// costs no accuracy that matters in FP64.
#include "common.cuh"

#include <algorithm>
#include <cmath>
#include <new>
#include <string>

using namespace rgsdev;

namespace {

constexpr int LZ = 512;          // threads of the cooperative kernels (one CTA per SM)
constexpr int NWZ = LZ / 32;
constexpr int kMaxM = 1024;

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

__device__ __forceinline__ double to_f64(double v) { return v; }
__device__ __forceinline__ double to_f64(float v) { return (double)v; }
__device__ __forceinline__ double to_f64(__nv_bfloat16 v) { return (double)__bfloat162float(v); }

// out(:, c) = V(:, c0 + c) * vscale[c0 + c] in FP64 (n rows, ld n), for the sketches of V.
template <typename TQ>
__global__ void scaled_copy_kernel(const TQ* V, int64_t ldv, const double* vscale, int64_t n, int c0, double* out) {
    const int c = blockIdx.y;
    const double s = vscale ? vscale[c0 + c] : 1.0;
    const TQ* col = V + (int64_t)(c0 + c) * ldv;
    double* o = out + (int64_t)c * n;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
        o[r] = to_f64(col[r]) * s;
}

// G = A^T A (m x m, ld m) for A k x m (ld lda): one 32 x 32 tile of the lower triangle per CTA of
// 32 x 8 threads (each thread four entries), 32 rows of A at a time through shared memory; the
// tile is written to both triangles (G exactly symmetric).
__global__ void __launch_bounds__(256) gram_kernel(const double* A, int64_t lda, int k, int m, double* G) {
    const int bi = blockIdx.y, bj = blockIdx.x;
    if (bj > bi) return;
    __shared__ double As[32][33], Bs[32][33];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int I0 = bi * 32, J0 = bj * 32;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (int l0 = 0; l0 < k; l0 += 32) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int c = ty + 8 * q, l = l0 + tx;
            As[tx][c] = (l < k && I0 + c < m) ? A[l + (int64_t)(I0 + c) * lda] : 0.0;
            Bs[tx][c] = (l < k && J0 + c < m) ? A[l + (int64_t)(J0 + c) * lda] : 0.0;
        }
        __syncthreads();
#pragma unroll 8
        for (int l = 0; l < 32; ++l) {
            const double b = Bs[l][tx];
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] = fma(As[l][ty + 8 * q], b, acc[q]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int i = I0 + ty + 8 * q, j = J0 + tx;
        if (i < m && j < m) {
            G[i + (int64_t)j * m] = acc[q];
            G[j + (int64_t)i * m] = acc[q];
        }
    }
}

// In-place right-looking Cholesky of the SPD matrix G (m x m, ld m; lower triangle used):
// step j subtracts G(i, j) G(l, j) / G(j, j) from G(i, l) for m > i >= l > j (a warp per column l,
// lanes over rows), then a grid barrier.  Afterwards LT(t, i) = L(i, t) = G(i, t) / sqrt(G(t, t)) for
// t <= i: row i of L is contiguous in LT.  Entries written by other SMs are read past L1
// (__ldcg).  A pivot that is not positive (or not finite) sets flag[0] = 1 and every CTA leaves.
__global__ void __launch_bounds__(LZ, 1) chol_kernel(double* G, int m, double* LT, int* ctl, int* flag) {
    pdl_wait();
    GridBarrier bar(ctl);
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x + gridDim.x * (threadIdx.x >> 5), nw = gridDim.x * NWZ;
    for (int j = 0; j < m; ++j) {
        const double d = __ldcg(G + j + (int64_t)j * m);
        if (!(d > 0.0) || !isfinite(d)) {                  // the same value in every CTA
            if (blockIdx.x == 0 && threadIdx.x == 0) flag[0] = 1;
            return;
        }
        const double inv = 1.0 / d;
        for (int l = j + 1 + gw; l < m; l += nw) {
            const double glj = __ldcg(G + l + (int64_t)j * m) * inv;
            double* gl = G + (int64_t)l * m;
            const double* gj = G + (int64_t)j * m;
            for (int i = l + lane; i < m; i += 32) gl[i] = __ldcg(gl + i) - __ldcg(gj + i) * glj;
        }
        if (!bar.sync(ctl)) return;
    }
    const int gtid = blockIdx.x * LZ + threadIdx.x, nth = gridDim.x * LZ;
    for (int64_t e = gtid; e < (int64_t)m * m; e += nth) {
        const int i = (int)(e / m), t = (int)(e % m);           // LT(t, i) = L(i, t)
        LT[e] = t <= i ? __ldcg(G + i + (int64_t)t * m) / sqrt(__ldcg(G + t + (int64_t)t * m)) : 0.0;
    }
}

// X(:, c) = L^{-1} b_c for the columns c of a right-hand side b_c(i) = B[i * bsr + c * bsc]
// (forward substitution, a warp per column, the solution in shared memory; L given as LT, row i
// of L contiguous).  Four warps per CTA.
__global__ void __launch_bounds__(128) trsv_cols_kernel(const double* LT, int m, const double* B, int64_t bsr,
                                                        int64_t bsc, double* X) {
    extern __shared__ double sx[];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c = blockIdx.x * 4 + w;
    if (c >= m) return;
    double* x = sx + (size_t)w * m;
    for (int i = 0; i < m; ++i) {
        const double* lrow = LT + (int64_t)i * m;
        double s0 = 0.0, s1 = 0.0;
        int t = lane;
        for (; t + 32 < i; t += 64) {
            s0 = fma(lrow[t], x[t], s0);
            s1 = fma(lrow[t + 32], x[t + 32], s1);
        }
        if (t < i) s0 = fma(lrow[t], x[t], s0);
        const double s = warp_sum(s0 + s1);
        const double v = (B[(int64_t)i * bsr + (int64_t)c * bsc] - s) / lrow[i];
        if (lane == 0) x[i] = v;
        __syncwarp();
    }
    for (int i = lane; i < m; i += 32) X[i + (int64_t)c * m] = x[i];
}

// Cs = (C + C^T) / 2 (m x m, ld m).
__global__ void symmetrize_kernel(const double* C, int m, double* Cs) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)m * m) return;
    const int i = (int)(e % m), j = (int)(e / m);
    Cs[e] = 0.5 * (C[i + (int64_t)j * m] + C[j + (int64_t)i * m]);
}

// Entry i of the Lanczos start vector: a standard normal from Philox4x32-10 (counter (i, 0, 0, 7),
// a fixed key), Box-Muller on two 53-bit uniforms.
__device__ double start_entry(int i) {
    uint32_t c[4] = {(uint32_t)i, 0u, 0u, 7u};
    philox4x32_10(c, 0x2545F491u, 0x9E3779B9u);
    const double u1 = u53(c[0], c[1]), u2 = u53(c[2], c[3]);
    return sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
}

struct LzParams {
    const double* C;      // m x m symmetric, ld m
    int m;
    double* Q;            // Lanczos vectors q_0..q_{m-1}, m x m, ld m
    double* w0;           // residual / product vectors (swapped every step)
    double* w1;
    double* h;            // Gram-Schmidt coefficients of the two passes
    double* h2;
    double* part;         // per-CTA sums of squares
    double* alpha;        // T's diagonal (m)
    double* beta;         // T's off-diagonal (m - 1)
    int* ctl;
};

// m Lanczos steps on C.  Step j: w = C q_j with q_j = r / beta_{j-1} formed in the same phase
// (q_0 the normalised start vector); two passes of classical Gram-Schmidt of w against
// q_0..q_j (coefficients h: a warp per vector; update: a thread per row); alpha_j is the sum of
// both passes' coefficients on q_j and beta_j = ||w||.  Five grid barriers per step.
__global__ void __launch_bounds__(LZ, 1) lanczos_kernel(LzParams p) {
    pdl_wait();
    GridBarrier bar(p.ctl);
    __shared__ double sh[NWZ + 1];
    __shared__ double sbeta;
    const int m = p.m;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gtid = blockIdx.x * LZ + threadIdx.x, nth = gridDim.x * LZ;
    const int gw = blockIdx.x + gridDim.x * warp, nw = gridDim.x * NWZ;
    double nrm0;
    {
        double ss = 0.0;
        for (int i = threadIdx.x; i < m; i += LZ) {
            const double g = start_entry(i);
            ss = fma(g, g, ss);
        }
        nrm0 = sqrt(block_sum<LZ>(ss, sh));           // the same value in every CTA
    }
    for (int j = 0; j < m; ++j) {
        double* wr = (j & 1) ? p.w1 : p.w0;          // residual of step j - 1
        double* wv = (j & 1) ? p.w0 : p.w1;          // this step's vector
        double qscale;                               // q_j = x * qscale, x = start vector or residual
        if (j == 0) {
            qscale = 1.0 / nrm0;
        } else {
            if (threadIdx.x < 32) {
                double s = 0.0;
                for (int b = lane; b < (int)gridDim.x; b += 32) s += __ldcg(p.part + b);
                s = warp_sum(s);
                if (lane == 0) sbeta = sqrt(s);
            }
            __syncthreads();
            const double beta = sbeta;
            if (gtid == 0) p.beta[j - 1] = beta;
            qscale = beta > 0.0 ? 1.0 / beta : 0.0;
        }
        // P1: q_j stored (thread per row) and w = C q_j (warp per row; column i of C = row i)
        double* qj = p.Q + (int64_t)j * m;
        for (int i = gtid; i < m; i += nth) qj[i] = (j == 0 ? start_entry(i) : __ldcg(wr + i)) * qscale;
        for (int i = gw; i < m; i += nw) {
            const double* ci = p.C + (int64_t)i * m;
            double s0 = 0.0, s1 = 0.0;
            for (int t = lane; t < m; t += 64) {
                const double x0 = j == 0 ? start_entry(t) : __ldcg(wr + t);
                s0 = fma(ci[t], x0, s0);
                if (t + 32 < m) {
                    const double x1 = j == 0 ? start_entry(t + 32) : __ldcg(wr + t + 32);
                    s1 = fma(ci[t + 32], x1, s1);
                }
            }
            const double s = warp_sum(s0 + s1);
            if (lane == 0) wv[i] = s * qscale;
        }
        if (!bar.sync(p.ctl)) return;
        for (int pass = 0; pass < 2; ++pass) {
            double* hh = pass == 0 ? p.h : p.h2;
            for (int t = gw; t <= j; t += nw) {           // hh[t] = q_t . w
                const double* qt = p.Q + (int64_t)t * m;
                double s0 = 0.0, s1 = 0.0;
                for (int i = lane; i < m; i += 64) {
                    s0 = fma(__ldcg(qt + i), __ldcg(wv + i), s0);
                    if (i + 32 < m) s1 = fma(__ldcg(qt + i + 32), __ldcg(wv + i + 32), s1);
                }
                const double s = warp_sum(s0 + s1);
                if (lane == 0) hh[t] = s;
            }
            if (!bar.sync(p.ctl)) return;
            double ss = 0.0;                                // w -= Q(:, 0:j) hh
            for (int i = gtid; i < m; i += nth) {
                double v = __ldcg(wv + i);
                for (int t = 0; t <= j; ++t) v = fma(-__ldcg(p.Q + i + (int64_t)t * m), __ldcg(hh + t), v);
                wv[i] = v;
                ss = fma(v, v, ss);
            }
            if (pass == 1) {
                ss = block_sum<LZ>(ss, sh);
                if (threadIdx.x == 0) p.part[blockIdx.x] = ss;
                if (gtid == 0) p.alpha[j] = __ldcg(p.h + j) + __ldcg(p.h2 + j);
            }
            if (!bar.sync(p.ctl)) return;
        }
    }
}

// Number of eigenvalues below x of the symmetric tridiagonal matrix with diagonal a and squared
// off-diagonal b2 (Sturm count from the LDL^T pivots; an exact zero pivot is moved just below 0).
__device__ int sturm_count(const double* a, const double* b2, int m, double x, double tiny) {
    int cnt = 0;
    double d = a[0] - x;
    if (d == 0.0) d = -tiny;
    cnt += d < 0.0;
    for (int i = 1; i < m; ++i) {
        d = (a[i] - x) - b2[i - 1] / d;
        if (d == 0.0) d = -tiny;
        cnt += d < 0.0;
    }
    return cnt;
}

// The smallest and the largest eigenvalue of T (alpha[0..m), beta[0..m-1)) by multisection:
// threads 0-255 bracket lambda_min, 256-511 lambda_max; every round each thread counts the
// eigenvalues below one of 256 interior points of its bracket and the bracket shrinks to one of
// the 257 pieces (eight rounds from the Gershgorin interval).  out = {lower end of the lambda_min
// bracket, upper end of the lambda_max bracket}.
__global__ void __launch_bounds__(512) tridiag_extremes_kernel(const double* alpha, const double* beta, int m,
                                                               double* out) {
    __shared__ double sa[kMaxM], sb2[kMaxM];
    __shared__ double lo[2], hi[2];
    __shared__ int cnt[512];
    for (int i = threadIdx.x; i < m; i += 512) {
        sa[i] = alpha[i];
        sb2[i] = i + 1 < m ? beta[i] * beta[i] : 0.0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double L = INFINITY, H = -INFINITY;
        for (int i = 0; i < m; ++i) {
            const double r = (i > 0 ? fabs(beta[i - 1]) : 0.0) + (i + 1 < m ? fabs(beta[i]) : 0.0);
            L = fmin(L, sa[i] - r);
            H = fmax(H, sa[i] + r);
        }
        const double pad = 1e-12 * fmax(fabs(L), fabs(H)) + 1e-300;
        lo[0] = lo[1] = L - pad;
        hi[0] = hi[1] = H + pad;
    }
    __syncthreads();
    const double tiny = 1e-300;
    const int g = threadIdx.x >> 8, r = threadIdx.x & 255;
    const int target = g == 0 ? 1 : m;
    for (int it = 0; it < 8; ++it) {
        const double L = lo[g], H = hi[g];
        cnt[threadIdx.x] = sturm_count(sa, sb2, m, L + (H - L) * (double)(r + 1) / 257.0, tiny);
        __syncthreads();
        if (r == 0) {
            int f = 256;                                  // first point with count >= target
            for (int q = 0; q < 256; ++q)
                if (cnt[g * 256 + q] >= target) { f = q; break; }
            lo[g] = f == 0 ? L : L + (H - L) * (double)f / 257.0;
            hi[g] = f == 256 ? H : L + (H - L) * (double)(f + 1) / 257.0;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = lo[0];
        out[1] = hi[1];
    }
}

}  // namespace

extern "C" rgs_status rgs_certify_embedding(rgs_handle h, rgs_sketch theta, rgs_sketch phi, int64_t n, int32_t m,
                                            const void* V, rgs_dtype vtype, int64_t ldv, const double* vscale,
                                            const double* VTheta, int64_t ldvt, double eps_star, double* out) {
    if (!h || !theta || !phi || !out) return RGS_ERR_INVALID_ARG;
    bool no_cert = false;
    const rgs_status st = guarded(h, [&] {
        RGS_REQUIRE(vtype == RGS_F64 || vtype == RGS_F32 || vtype == RGS_BF16, "unknown vtype");
        RGS_REQUIRE(theta->n == n && phi->n == n, "n differs from the sketches' n");
        RGS_REQUIRE(m >= 1 && m <= kMaxM && m <= theta->k && m <= phi->k, "need 1 <= m <= min(1024, k_theta, k_phi)");
        RGS_REQUIRE(V != nullptr && ldv >= n, "null V or ldv < n");
        RGS_REQUIRE(VTheta == nullptr || ldvt >= theta->k, "ldvt < k");
        RGS_REQUIRE(eps_star >= 0.0 && eps_star < 1.0, "need 0 <= eps_star < 1");
        RGS_REQUIRE(!rgs_is_host_pointer(V) && !rgs_is_host_pointer(vscale) && !rgs_is_host_pointer(VTheta),
                    "V, vscale and VTheta must be device pointers");
        const int kt = theta->k, kp = phi->k;
        const size_t mm = (size_t)m * m;
        // workspace: Phi V, Theta V (when not given), G_Phi, G_Theta, LT, B, C, Q, vectors
        size_t off = 0;
        auto take = [&](size_t cnt) { const size_t o = off; off += (cnt + 31) & ~(size_t)31; return o; };
        const size_t oYp = take((size_t)kp * m), oYt = take(VTheta ? 0 : (size_t)kt * m), oGp = take(mm),
                     oGt = take(mm), oLT = take(mm), oB = take(mm), oC = take(mm), oQ = take(mm),
                     ow0 = take(m), ow1 = take(m), oh = take(m), oh2 = take(m), opart = take(h->num_sms),
                     oal = take(m), obe = take(m), oex = take(2);
        h->cert.ensure(off * sizeof(double));
        double* b = h->cert.as<double>();
        double* Yp = b + oYp;
        double* Yt = VTheta ? nullptr : b + oYt;
        cudaStream_t s = h->stream;
        // the sketches of V's columns (scaled to FP64), in chunks of columns
        const int esz = vtype == RGS_F64 ? 8 : (vtype == RGS_F32 ? 4 : 2);
        const int cb = (int)std::max<int64_t>(1, std::min<int64_t>(m, ((int64_t)256 << 20) / (8 * n)));
        h->cert_cols.ensure(sizeof(double) * (size_t)n * cb);
        double* cols = h->cert_cols.as<double>();
        for (int c0 = 0; c0 < m; c0 += cb) {
            const int nc = std::min(cb, m - c0);
            const dim3 grid((unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 256)), nc);
            const char* vb = static_cast<const char*>(V);
            if (vtype == RGS_F64)
                scaled_copy_kernel<double><<<grid, 256, 0, s>>>(reinterpret_cast<const double*>(vb), ldv, vscale, n, c0, cols);
            else if (vtype == RGS_F32)
                scaled_copy_kernel<float><<<grid, 256, 0, s>>>(reinterpret_cast<const float*>(vb), ldv, vscale, n, c0, cols);
            else
                scaled_copy_kernel<__nv_bfloat16><<<grid, 256, 0, s>>>(reinterpret_cast<const __nv_bfloat16*>(vb), ldv,
                                                                       vscale, n, c0, cols);
            RGS_CUDA(cudaGetLastError());
            (void)esz;
            rgs_sketch_columns(h, phi, nc, cols, n, Yp + (size_t)c0 * kp, kp);
            if (Yt) rgs_sketch_columns(h, theta, nc, cols, n, Yt + (size_t)c0 * kt, kt);
        }
        const double* At = VTheta ? VTheta : Yt;
        const int64_t lat = VTheta ? ldvt : kt;
        const int nt = (m + 31) / 32;
        gram_kernel<<<dim3(nt, nt), dim3(32, 8), 0, s>>>(Yp, kp, kp, m, b + oGp);
        RGS_CUDA(cudaGetLastError());
        gram_kernel<<<dim3(nt, nt), dim3(32, 8), 0, s>>>(At, lat, kt, m, b + oGt);
        RGS_CUDA(cudaGetLastError());
        RGS_CUDA(cudaMemsetAsync(h->ctl.ptr, 0, kCtlWords * sizeof(int), s));
        int* ctl = h->ctl.as<int>();
        int* flag = ctl + kFlagWord;
        const int grid = h->num_sms;
        {
            double* G = b + oGp;
            double* LT = b + oLT;
            void* args[] = {&G, (void*)&m, &LT, &ctl, &flag};
            RGS_CUDA(cudaLaunchCooperativeKernel((const void*)chol_kernel, dim3(grid), dim3(LZ), args, 0, s));
        }
        const size_t tsm = 4 * sizeof(double) * (size_t)m;
        trsv_cols_kernel<<<(m + 3) / 4, 128, tsm, s>>>(b + oLT, m, b + oGt, 1, m, b + oB);      // B = L^{-1} G_Theta
        RGS_CUDA(cudaGetLastError());
        trsv_cols_kernel<<<(m + 3) / 4, 128, tsm, s>>>(b + oLT, m, b + oB, m, 1, b + oC);      // C = L^{-1} B^T
        RGS_CUDA(cudaGetLastError());
        symmetrize_kernel<<<(unsigned)((mm + 255) / 256), 256, 0, s>>>(b + oC, m, b + oB);   // symmetric C in B
        RGS_CUDA(cudaGetLastError());
        {
            LzParams p{};
            p.C = b + oB;
            p.m = m;
            p.Q = b + oQ;
            p.w0 = b + ow0;
            p.w1 = b + ow1;
            p.h = b + oh;
            p.h2 = b + oh2;
            p.part = b + opart;
            p.alpha = b + oal;
            p.beta = b + obe;
            p.ctl = ctl;
            void* args[] = {&p};
            RGS_CUDA(cudaLaunchCooperativeKernel((const void*)lanczos_kernel, dim3(grid), dim3(LZ), args, 0, s));
        }
        tridiag_extremes_kernel<<<1, 512, 0, s>>>(b + oal, b + obe, m, b + oex);
        RGS_CUDA(cudaGetLastError());
        h->launches += 8;
        double ex[2];
        int ctlv[kCtlWords];
        RGS_CUDA(cudaMemcpyAsync(ex, b + oex, sizeof(ex), cudaMemcpyDeviceToHost, s));
        RGS_CUDA(cudaMemcpyAsync(ctlv, h->ctl.ptr, sizeof(ctlv), cudaMemcpyDeviceToHost, s));
        RGS_CUDA(cudaStreamSynchronize(s));
        if (ctlv[kStatusWord] != 0)
            throw RgsError{(rgs_status)ctlv[kStatusWord], std::string("device status in the certificate: ") +
                                                              rgs_status_string((rgs_status)ctlv[kStatusWord])};
        if (ctlv[kFlagWord] != 0)
            throw RgsError{RGS_ERR_NONFINITE, "the Gram matrix of Phi V is not numerically positive definite"};
        const double lmin = std::max(ex[0], 0.0), lmax = ex[1];
        const double wb = std::max(1.0 - (1.0 - eps_star) * lmin, (1.0 + eps_star) * lmax - 1.0);
        out[0] = wb;
        out[1] = std::sqrt(lmin);
        out[2] = std::sqrt(lmax);
        no_cert = !(wb < 1.0);
    });
    if (st == RGS_OK && no_cert) {
        h->last_error = "omega_bar >= 1: no embedding certificate";
        return RGS_ERR_CERT_FAILED;
    }
    return st;
}
