// Alg. 2 steps 2, 5, 6 on the GPU in FP64: the sketched least-squares problem
// argmin_y ||S_{i-1} y - p_i|| solved through a Householder QR of S (the solver
// of the paper's experiments, Sec. 5), kept incrementally in compact-WY form
//     H_0 H_1 ... H_{i-1} = I - V T V^T,    S_i = (H_0 ... H_{i-1}) [R_S; 0],
// together with M = V T and R_S^{-1}.  With that form every phase is a parallel matrix-vector
// product spread over the whole GPU instead of i dependent reflector applications:
//   y  = [s, p] - V (M^T [s, p])         (apply the i existing reflectors: I - V T^T V^T)
//   new reflector H_i from y_s(i:k)      (appends s_i, column i of R_S = [y_s(0:i); beta])
//   x  = R_S^{-1} (H_i y_p)(0:i+1)       (the least-squares solution)
//   T(0:i, i) = -tau_i T V^T v_i, R_S^{-1} gains the column -R_S^{-1} y_s(0:i) / beta,
//   M(:, i) = V T(:, i) (formed at the start of the next launch).
// One cooperative launch per column; phases are separated by bounded grid barriers.  GB300 runs
// FP64 at 2 operations per clock per SM and an L2 round trip costs about a microsecond, so the
// phases are arranged to keep dependent round trips and redundant FP64 scalar work short.
#include "common.cuh"
#include "givens.cuh"

#include <algorithm>

using namespace rgsdev;

namespace {

constexpr int LT = 512;        // threads per CTA (one CTA per SM)
constexpr int NW = LT / 32;    // warps per CTA
constexpr int GS = 32;         // partial sketches summed per warp in the first reduction level

__device__ __forceinline__ double ldcg(const double* p) { return __ldcg(p); }

// Block-wide sums of N values at once (trees: shuffles within warps, then one warp),
// identical in every thread; sm holds at least N * (NW + 1) doubles.
template <int N>
__device__ __forceinline__ void block_sum_n(double (&v)[N], double* sm) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < N; ++q) v[q] = warp_sum(v[q]);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < N; ++q) sm[q * NW + w] = v[q];
    __syncthreads();
    if (threadIdx.x < 32) {
#pragma unroll
        for (int q = 0; q < N; ++q) {
            double t = lane < NW ? sm[q * NW + lane] : 0.0;
            t = warp_sum(t);
            if (lane == 0) sm[N * NW + q] = t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < N; ++q) v[q] = sm[N * NW + q];
}

// Block-wide sums of N values held by lane 0 of each warp (other lanes ignored): one warp
// adds the NW per-warp values, so only NW/32-wide FP64 work is spent on the reduction.
template <int N>
__device__ __forceinline__ void block_sum_lane0(double (&v)[N], double* sm) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < N; ++q) sm[q * NW + w] = v[q];
    __syncthreads();
    if (threadIdx.x < 32) {
#pragma unroll
        for (int q = 0; q < N; ++q) {
            double t = lane < NW ? sm[q * NW + lane] : 0.0;
            t = warp_sum(t);
            if (lane == 0) sm[N * NW + q] = t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < N; ++q) v[q] = sm[N * NW + q];
}

constexpr int kTotMax = 8;     // grid_total2 reads up to 32 * kTotMax CTAs' values in one round trip

// Deterministic totals of the per-CTA values blk[b*4 + off] and blk[b*4 + off + 1],
// identical in every CTA; one warp issues all the loads at once, does the FP64 adds and
// broadcasts through shared memory.
__device__ double2 grid_total2(const double* blk, int off, double* sh) {
    __syncthreads();
    if (threadIdx.x < 32) {
        const int G = gridDim.x;
        double a0[kTotMax], a1[kTotMax];
#pragma unroll
        for (int q = 0; q < kTotMax; ++q) {
            const int b = threadIdx.x + 32 * q;
            a0[q] = b < G ? ldcg(blk + (size_t)b * 4 + off) : 0.0;
            a1[q] = b < G ? ldcg(blk + (size_t)b * 4 + off + 1) : 0.0;
        }
        double v0 = 0.0, v1 = 0.0;
#pragma unroll
        for (int q = 0; q < kTotMax; ++q)
            if (32 * q < G) { v0 += a0[q]; v1 += a1[q]; }
        v0 = warp_sum(v0);
        v1 = warp_sum(v1);
        if (threadIdx.x == 0) { sh[0] = v0; sh[1] = v1; }
    }
    __syncthreads();
    const double2 t = make_double2(sh[0], sh[1]);
    __syncthreads();
    return t;
}

// Sum over b in [b0, b1) of src[b * k + l]: partial sketches (double-float or FP64) written by an
// earlier launch, or (CG) FP64 group sums written by this launch, read through L2.
template <bool CG = false>
__device__ __forceinline__ double group_sum(const double* src, bool sdf, int b0, int b1, int k, int l) {
    if (sdf) {
        const df* d = reinterpret_cast<const df*>(src);
        df t0 = {0.f, 0.f}, t1 = {0.f, 0.f};
        int b = b0;
#pragma unroll 16
        for (; b + 1 < b1; b += 2) {
            t0 = df_add(t0, d[(size_t)b * k + l]);
            t1 = df_add(t1, d[(size_t)(b + 1) * k + l]);
        }
        if (b < b1) t0 = df_add(t0, d[(size_t)b * k + l]);
        t0 = df_add(t0, t1);
        return (double)t0.h + (double)t0.l;
    }
    auto ld = [&](int b) { return CG ? ldcg(src + (size_t)b * k + l) : src[(size_t)b * k + l]; };
    double v0 = 0.0, v1 = 0.0, v2 = 0.0, v3 = 0.0;
    int b = b0;
#pragma unroll 2
    for (; b + 3 < b1; b += 4) {
        v0 += ld(b);
        v1 += ld(b + 1);
        v2 += ld(b + 2);
        v3 += ld(b + 3);
    }
    for (; b < b1; ++b) v0 += ld(b);
    return (v0 + v1) + (v2 + v3);
}

__global__ void __launch_bounds__(LT, 1) ls_kernel(LSState st, LSStep a) {
    __shared__ double sh[3 * (NW + 1) + 2 + 3 * NW];
    __shared__ double sc[8];
    int* ctl = st.ctl;
    if (ctl[kStatusWord] != 0 || ctl[kStopWord] != 0) return;
    const int k = st.k, mm = st.mmax, i = a.i;
    const int G = gridDim.x;
    const int tid = threadIdx.x, lane = tid & 31;
    const int nthreads = G * LT, gtid = blockIdx.x * LT + tid;
    // warp w of CTA b is global warp b + G*w, so consecutive items spread over all SMs
    const int gwarp = blockIdx.x + G * (tid >> 5), nwarps = nthreads >> 5;
    const bool app = a.append != 0, sol = a.solve != 0;
    const bool p_parts = sol && a.p_vec == nullptr;
    unsigned long long* trace = (a.trace != nullptr && blockIdx.x == 0 && tid == 0) ? a.trace : nullptr;
    if (trace) trace[0] = globaltimer();
    GridBarrier bar(ctl);
    const double pref = (app && tid == 0) ? st.pnorm[i] : 0.0;   // ||p_i||, for the breakdown test

    // ---- phase 0a: with more than GS partial sketches, a first level sums groups of GS
    const int sgroups = app ? (a.s_nparts + GS - 1) / GS : 0;
    const int pgroups = p_parts ? (a.p_nparts + GS - 1) / GS : 0;
    const bool level1 = sgroups > 1 || pgroups > 1;
    if (level1) {
        const int nseg = (k + 31) / 32;
        for (int it = gwarp; it < nseg * (sgroups + pgroups); it += nwarps) {
            const int seg = it % nseg, g = it / nseg;
            const bool is_s = g < sgroups;
            const int gg = is_s ? g : g - sgroups;
            const int np = is_s ? a.s_nparts : a.p_nparts;
            const int l = seg * 32 + lane;
            if (l < k)
                st.red[(size_t)g * k + l] = group_sum(is_s ? a.s_part : a.p_part, is_s ? a.s_df : a.p_df,
                                                      gg * GS, min(np, gg * GS + GS), k, l);
        }
        if (!bar.sync(ctl)) return;
    }
    if (trace) trace[1] = globaltimer();

    // ---- phase 0b: a warp per 32 rows (lane = row), each lane summing the groups (or partials)
    //      of its row in order: s', p and their squared norms
    {
        double nrm[2] = {0.0, 0.0};
        const int nseg = (k + 31) / 32;
        const bool busy = gwarp < nseg;
        for (int seg = gwarp; seg < nseg; seg += nwarps) {
            const int l = seg * 32 + lane;
            if (l >= k) continue;
            if (app) {
                const double v = (level1 ? group_sum<true>(st.red, false, 0, sgroups, k, l)
                                         : group_sum(a.s_part, a.s_df != 0, 0, a.s_nparts, k, l)) * a.s_scale;
                st.sbuf[l] = v;
                nrm[0] = fma(v, v, nrm[0]);
            }
            if (sol) {
                const double v = (!p_parts ? a.p_vec[l]
                                  : level1 ? group_sum<true>(st.red + (size_t)sgroups * k, false, 0, pgroups, k, l)
                                           : group_sum(a.p_part, a.p_df != 0, 0, a.p_nparts, k, l)) * a.p_scale;
                st.pbuf[l] = v;
                if (a.p_store) a.p_store[l] = v;
                nrm[1] = fma(v, v, nrm[1]);
            }
        }
        if (i > 0) {
            // M(:, i-1) = V(:, 0:i) T(0:i, i-1): T's column i-1 was completed by the previous
            // launch; warp per row of the row-major copy VT, lanes over the columns
            const double* tc = st.T + (size_t)(i - 1) * mm;
            for (int l = gwarp; l < k; l += nwarps) {
                const double* vr = st.VT + (size_t)l * mm;
                const int jend = min(i, l + 1);
                double acc[4] = {0.0, 0.0, 0.0, 0.0};
                int j = lane;
                for (; j + 96 < jend; j += 128)
#pragma unroll
                    for (int q = 0; q < 4; ++q) acc[q] = fma(vr[j + 32 * q], tc[j + 32 * q], acc[q]);
                for (; j < jend; j += 32) acc[0] = fma(vr[j], tc[j], acc[0]);
                const double d = warp_sum((acc[0] + acc[1]) + (acc[2] + acc[3]));
                if (lane == 0) st.M[(size_t)(i - 1) * k + l] = d;
            }
        }
        if (busy) {                                    // idle warps skip the FP64 shuffles
            nrm[0] = warp_sum(nrm[0]);
            nrm[1] = warp_sum(nrm[1]);
        }
        block_sum_lane0<2>(nrm, sh);
        if (tid == 0) { st.blk[blockIdx.x * 4 + 0] = nrm[0]; st.blk[blockIdx.x * 4 + 1] = nrm[1]; }
    }
    if (!bar.sync(ctl)) return;
    if (trace) trace[2] = globaltimer();

    // ---- phase 1: r_ii, s_i = s'/r_ii; u2 = M(:, 0:i)^T [s, p] = T^T V^T [s, p]
    const double2 tot01 = grid_total2(st.blk, 0, sh);
    // The phase's scalars come from one thread through shared memory: an FP64 square root or
    // division is a long sequence on the FP64 pipe, which would otherwise run in every thread.
    if (tid == 0) {
        const double r0 = sqrt(tot01.x);
        int code = 0;                                  // 1: non-finite r_ii, 2: breakdown
        if (app) code = !isfinite(r0) ? 1 : (!(r0 > 16.0 * 0x1p-53 * pref) ? 2 : 0);
        const double ir = code == 0 ? 1.0 / r0 : 1.0;
        sc[0] = r0;
        sc[1] = app ? ir : 1.0;
        sc[2] = (app && a.p_lag) ? ir : 1.0;
        sc[3] = sol ? sqrt(tot01.y) : 0.0;
        sc[4] = (double)code;
    }
    __syncthreads();
    const double r = sc[0], pn = sc[3];
    const int code = (int)sc[4];
    double inv_r = 1.0, pmul = 1.0;
    if (app) {
        if (code == 1) {
            if (gtid == 0) { atomicCAS(ctl + kStatusWord, 0, (int)RGS_ERR_NONFINITE); ctl[kDetailWord] = i; }
            return;
        }
        const bool breakdown = code == 2;
        if (a.givens) {
            // GMRES: H(:, i-1) = R(0:i+1, i) (Sec. 4.1) is complete now that r_ii is known
            if (i == 0) {
                if (gtid == 0) st.g[0] = r;
            } else if (blockIdx.x == G - 1 && tid < 32) {
                const double* rc = st.R + (size_t)i * st.ldr;
                auto hcol = [&](int t) { return t < i ? rc[t] : r; };
                const double res = givens_column_warp(i - 1, hcol, st.cs, st.sn, st.g, st.Hr, mm);
                if (tid == 0 && (breakdown || res <= a.stop_tol)) atomicCAS(ctl + kStopWord, 0, i);
            }
        }
        if (breakdown) {
            if (!(a.arnoldi && i > 0) && gtid == 0) {
                atomicCAS(ctl + kStatusWord, 0, (int)RGS_ERR_BREAKDOWN);
                ctl[kDetailWord] = i;
            }
            return;
        }
        inv_r = sc[1];
        pmul = sc[2];
        if (gtid == 0) {
            st.R[(size_t)i * st.ldr + i] = r;
            st.sigma[i] = inv_r;
        }
    }
    if (sol && gtid == 0) st.pnorm[a.pnorm_idx] = pn * pmul;
    {
        // a quad of warps (one per SM sub-partition) per column; each warp a quarter of the rows
        const int quad = tid >> 7, qw = (tid >> 5) & 3;
        double* qs = sh + 3 * (NW + 1) + 2;                // [NW/4 quads][4 warps][2]
        const int seg = (k + 3) / 4;
        for (int base = 0; base < i; base += G * (NW / 4)) {
            const int j = base + blockIdx.x + G * quad;
            double ds = 0.0, dp = 0.0;
            if (j < i) {
                const double* mc = st.M + (size_t)j * k;      // column i-1 was written by phase 0b
                const int l0 = qw * seg, l1 = min(k, l0 + seg);
#pragma unroll 8
                for (int l = l0 + lane; l < l1; l += 32) {
                    const double mv = ldcg(mc + l);
                    if (app) ds = fma(mv, ldcg(st.sbuf + l), ds);
                    if (sol) dp = fma(mv, ldcg(st.pbuf + l), dp);
                }
                ds = warp_sum(ds);
                dp = warp_sum(dp);
                if (lane == 0) { qs[(quad * 4 + qw) * 2] = ds; qs[(quad * 4 + qw) * 2 + 1] = dp; }
            }
            __syncthreads();
            if (j < i && qw == 0 && lane == 0) {
                const double* q4 = qs + quad * 8;
                st.u2s[j] = ((q4[0] + q4[2]) + (q4[4] + q4[6])) * inv_r;
                st.u2p[j] = ((q4[1] + q4[3]) + (q4[5] + q4[7])) * pmul;
            }
            __syncthreads();
        }
    }
    if (!bar.sync(ctl)) return;
    if (trace) trace[3] = globaltimer();

    if (trace) trace[4] = trace[3];                  // (no separate T^T u phase: M holds V T)

    // ---- phase 3: y = [s, p] - V u2 (the i reflectors applied), warp per row using the
    //      row-major copy VT of V; plus the sums the new reflector needs over rows > i
    const int krows = app ? k : i;                 // a pure solve needs rows 0..i-1 only
    {
        double sums[2] = {0.0, 0.0};
        for (int l = gwarp; l < krows; l += nwarps) {
            const double* vr = st.VT + (size_t)l * mm;
            const int jend = min(i, l + 1);
            double as[4] = {0.0, 0.0, 0.0, 0.0}, ap[4] = {0.0, 0.0, 0.0, 0.0};
            int j = lane;
            for (; j + 96 < jend; j += 128)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const double vv = vr[j + 32 * q];
                    if (app) as[q] = fma(vv, ldcg(st.u2s + j + 32 * q), as[q]);
                    if (sol) ap[q] = fma(vv, ldcg(st.u2p + j + 32 * q), ap[q]);
                }
            for (; j < jend; j += 32) {
                const double vv = vr[j];
                if (app) as[0] = fma(vv, ldcg(st.u2s + j), as[0]);
                if (sol) ap[0] = fma(vv, ldcg(st.u2p + j), ap[0]);
            }
            const double ws = warp_sum((as[0] + as[1]) + (as[2] + as[3]));
            const double wp = warp_sum((ap[0] + ap[1]) + (ap[2] + ap[3]));
            if (lane == 0) {
                const double sl = app ? ldcg(st.sbuf + l) * inv_r : 0.0;
                if (app) st.S[(size_t)i * k + l] = sl;     // s_i (Alg. 2 step 6)
                const double ysl = app ? sl - ws : 0.0;
                const double ypl = sol ? ldcg(st.pbuf + l) * pmul - wp : 0.0;
                st.ys[l] = ysl;
                st.yp[l] = ypl;
                if (app && l > i) { sums[0] = fma(ysl, ysl, sums[0]); sums[1] = fma(ysl, ypl, sums[1]); }
            }
        }
        block_sum_lane0<2>(sums, sh);
        if (tid == 0) { st.blk[blockIdx.x * 4 + 2] = sums[0]; st.blk[blockIdx.x * 4 + 3] = sums[1]; }
    }
    if (!bar.sync(ctl)) return;
    if (trace) trace[5] = globaltimer();

    if (!app) {
        // pure solve: x = R_S^{-1} y(0:i); row j of R_S^{-1} is column j of RinvT
        for (int j = gwarp; j < i; j += nwarps) {
            const double* rr = st.RinvT + (size_t)j * mm;
            double da = 0.0, db = 0.0;
            int l = j + lane;
            for (; l + 32 < i; l += 64) {
                da = fma(rr[l], ldcg(st.yp + l), da);
                db = fma(rr[l + 32], ldcg(st.yp + l + 32), db);
            }
            if (l < i) da = fma(rr[l], ldcg(st.yp + l), da);
            const double d = warp_sum(da + db);
            if (lane == 0) {
                st.R[(size_t)a.xcol * st.ldr + j] = d;
                st.coef[j] = d * st.sigma[j];
            }
        }
        if (trace) { trace[6] = globaltimer(); trace[7] = trace[6]; }
        return;
    }

    // ---- phase 4: per column j < i, the dots the new reflector needs that do not depend on beta:
    //   zp_j = sum_{l>i} V(l,j) ys_l,  d1_j = sum_{j<=l<i} Rinv(j,l) ys_l,  d2_j likewise with yp
    {
        const int quad = tid >> 7, qw = (tid >> 5) & 3;
        double* qs = sh + 3 * (NW + 1) + 2;                // [NW/4 quads][4 warps][3]
        for (int base = 0; base < i; base += G * (NW / 4)) {
            const int j = base + blockIdx.x + G * quad;
            double z = 0.0, d1 = 0.0, d2 = 0.0;
            if (j < i) {
                const double* v = st.V + (size_t)j * k;
                const int len = k - (i + 1), seg = (max(len, 0) + 3) / 4;
                const int l0 = i + 1 + qw * seg, l1 = min(k, l0 + seg);
#pragma unroll 4
                for (int l = l0 + lane; l < l1; l += 32) z = fma(v[l], ldcg(st.ys + l), z);
                const double* rr = st.RinvT + (size_t)j * mm;       // row j of R_S^{-1}
                const int rlen = i - j, rseg = (rlen + 3) / 4;
                const int r0 = j + qw * rseg, r1 = min(i, r0 + rseg);
                for (int l = r0 + lane; l < r1; l += 32) {
                    const double rv = rr[l];
                    d1 = fma(rv, ldcg(st.ys + l), d1);
                    if (sol) d2 = fma(rv, ldcg(st.yp + l), d2);
                }
                z = warp_sum(z);
                d1 = warp_sum(d1);
                if (sol) d2 = warp_sum(d2);
                if (lane == 0) {
                    qs[(quad * 4 + qw) * 3] = z;
                    qs[(quad * 4 + qw) * 3 + 1] = d1;
                    qs[(quad * 4 + qw) * 3 + 2] = d2;
                }
            }
            __syncthreads();
            if (j < i && qw == 0 && lane == 0) {
                const double* q4 = qs + quad * 12;
                st.zp[j] = (q4[0] + q4[3]) + (q4[6] + q4[9]);
                st.d1[j] = (q4[1] + q4[4]) + (q4[7] + q4[10]);
                st.d2[j] = (q4[2] + q4[5]) + (q4[8] + q4[11]);
            }
            __syncthreads();
        }
    }
    if (!bar.sync(ctl)) return;
    if (trace) trace[6] = globaltimer();

    // ---- phase 5: the reflector H_i, V(:, i), T(0:i, i), R_S^{-1}(:, i) and x
    double alpha = 0.0, ypi0 = 0.0;
    if (tid == 0) {                                    // issued before the totals' round trip
        alpha = ldcg(st.ys + i);
        ypi0 = sol ? ldcg(st.yp + i) : 0.0;
    }
    const double2 tot23 = grid_total2(st.blk, 2, sh);
    const double SG = tot23.x, CR = tot23.y;
    if (tid == 0) {
        double beta, tau, vs;
        if (SG == 0.0) {
            beta = alpha; tau = 0.0; vs = 0.0;
        } else {
            const double nrm = sqrt(alpha * alpha + SG);
            beta = alpha >= 0.0 ? -nrm : nrm;
            tau = (beta - alpha) / beta;
            vs = 1.0 / (alpha - beta);
        }
        sc[0] = beta; sc[1] = tau; sc[2] = vs;
        sc[3] = sol ? ypi0 - tau * (ypi0 + CR * vs) : 0.0;
    }
    __syncthreads();
    const double beta = sc[0], tau = sc[1], vs = sc[2], ypi = sc[3];
    if (beta == 0.0) {
        if (gtid == 0) { atomicCAS(ctl + kStatusWord, 0, (int)RGS_ERR_BREAKDOWN); ctl[kDetailWord] = i; }
        return;
    }
    for (int l = gtid; l < k; l += nthreads) {
        const double vl = l < i ? 0.0 : (l == i ? 1.0 : ldcg(st.ys + l) * vs);
        st.V[(size_t)i * k + l] = vl;
        if (l >= i) st.VT[(size_t)l * mm + i] = vl;
    }
    if (gtid == 0) {
        st.T[(size_t)i * mm + i] = tau;
        st.TT[(size_t)i * mm + i] = tau;
        st.RinvT[(size_t)i * mm + i] = 1.0 / beta;
        if (sol) {
            const double xi = ypi / beta;
            st.R[(size_t)a.xcol * st.ldr + i] = xi;
            st.coef[i] = xi * inv_r;
        }
    }
    const double* vrow_i = st.VT + (size_t)i * mm;     // V(i, 0:i)
    for (int j = gwarp; j < i; j += nwarps) {
        // T(j, i) = -tau sum_{j<=l<i} T(j,l) z_l with z_l = V(i,l) + vs zp_l
        const double* tr = st.TT + (size_t)j * mm;
        double da = 0.0, db = 0.0;
        int l = j + lane;
        for (; l + 32 < i; l += 64) {
            da = fma(tr[l], vrow_i[l] + vs * ldcg(st.zp + l), da);
            db = fma(tr[l + 32], vrow_i[l + 32] + vs * ldcg(st.zp + l + 32), db);
        }
        if (l < i) da = fma(tr[l], vrow_i[l] + vs * ldcg(st.zp + l), da);
        const double d = warp_sum(da + db);
        if (lane == 0) {
            const double t = -tau * d;
            st.T[(size_t)i * mm + j] = t;
            st.TT[(size_t)j * mm + i] = t;
            const double cnew = -ldcg(st.d1 + j) / beta;       // R_S^{-1}(j, i)
            st.RinvT[(size_t)j * mm + i] = cnew;
            if (sol) {
                const double xj = ldcg(st.d2 + j) + cnew * ypi;
                st.R[(size_t)a.xcol * st.ldr + j] = xj;
                st.coef[j] = xj * st.sigma[j];
            }
        }
    }
    if (trace) trace[7] = globaltimer();
}

// Step 8 certificates: Delta_m = ||I - S^T S||_F, Delta~_m = ||P - S R||_F / ||P||_F.
// Block b handles column b: sums of squares of (I - S^T S)(0:m, b) and (P - S R)(:, b).
__global__ void __launch_bounds__(256) cert_kernel(const double* S, int k, int m, const double* R, int64_t ldr,
                                                   const double* P, double* work) {
    __shared__ double sh[256];
    const int b = blockIdx.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    double g2 = 0.0;
    for (int a = w; a < m; a += 8) {
        double d = 0.0;
        for (int l = lane; l < k; l += 32) d = fma(S[(size_t)a * k + l], S[(size_t)b * k + l], d);
        d = warp_sum(d);
        const double e = (a == b ? 1.0 : 0.0) - d;
        g2 += lane == 0 ? e * e : 0.0;
    }
    double e2 = 0.0, p2 = 0.0;
    for (int l = threadIdx.x; l < k; l += 256) {
        double v = P[(size_t)b * k + l];
        p2 += v * v;
        for (int j = 0; j <= b; ++j) v = fma(-S[(size_t)j * k + l], R[(size_t)b * ldr + j], v);
        e2 += v * v;
    }
    g2 = block_sum<256>(g2, sh);
    e2 = block_sum<256>(e2, sh);
    p2 = block_sum<256>(p2, sh);
    if (threadIdx.x == 0) { work[3 * b] = g2; work[3 * b + 1] = e2; work[3 * b + 2] = p2; }
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

void rgs_ls_alloc(DevBuf& buf, int k, int mmax, int grid, int max_parts, LSState* st) {
    const int groups = 2 * ((std::max(max_parts, 1) + GS - 1) / GS);
    size_t n = 0;
    auto take = [&](size_t cnt) { size_t off = n; n += (cnt + 31) & ~(size_t)31; return off; };
    const size_t oV = take((size_t)k * mmax), oVT = take((size_t)k * mmax), oT = take((size_t)mmax * mmax),
                 oTT = take((size_t)mmax * mmax), oRi = take((size_t)mmax * mmax), oS = take((size_t)k * mmax),
                 osb = take(k), opb = take(k), oys = take(k), oyp = take(k), oM = take((size_t)k * mmax),
                 ou2s = take(mmax), ou2p = take(mmax), ozp = take(mmax), od1 = take(mmax), od2 = take(mmax),
                 ored = take((size_t)groups * k), oblk = take((size_t)4 * grid), osg = take(mmax + 1),
                 opn = take(mmax + 2), oco = take(mmax + 1);
    buf.ensure(n * sizeof(double));
    double* b = buf.as<double>();
    st->k = k; st->mmax = mmax; st->max_parts = max_parts;
    st->V = b + oV; st->VT = b + oVT; st->T = b + oT; st->TT = b + oTT; st->RinvT = b + oRi; st->S = b + oS;
    st->sbuf = b + osb; st->pbuf = b + opb; st->ys = b + oys; st->yp = b + oyp;
    st->M = b + oM; st->u2s = b + ou2s; st->u2p = b + ou2p;
    st->zp = b + ozp; st->d1 = b + od1; st->d2 = b + od2;
    st->red = b + ored; st->blk = b + oblk; st->sigma = b + osg; st->pnorm = b + opn;
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
}

void rgs_launch_ls(rgs_context* ctx, const LSState& st, const LSStep& a) {
    RGS_REQUIRE(a.s_nparts <= st.max_parts && a.p_nparts <= st.max_parts, "too many partial sketches");
    LSState s = st;
    LSStep p = a;
    void* args[] = {&s, &p};
    const int grid = ctx->ls_blocks_tuned > 0 ? std::min(ctx->ls_blocks_tuned, ctx->ls_blocks) : ctx->ls_blocks;
    RGS_REQUIRE(grid <= 32 * kTotMax, "least-squares grid larger than the per-CTA totals support");
    RGS_CUDA(cudaLaunchCooperativeKernel((const void*)ls_kernel, dim3(grid), dim3(LT), args, 0, ctx->stream));
    ctx->launches++;
}

// One CTA of LT threads per SM (its registers fill the SM), so the cooperative grid is the SM count.
int rgs_ls_max_blocks(int num_sms) {
    int per_sm = 0;
    RGS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ls_kernel, LT, 0));
    RGS_REQUIRE(per_sm >= 1, "the least-squares kernel does not fit on an SM");
    return num_sms;
}

void rgs_launch_certificates(rgs_context* ctx, const double* S, int k, int m, const double* R, int64_t ldr,
                             const double* P, double* out2, double* work) {
    cert_kernel<<<m, 256, 0, ctx->stream>>>(S, k, m, R, ldr, P, work);
    RGS_CUDA(cudaGetLastError());
    cert_final_kernel<<<1, 256, 0, ctx->stream>>>(work, m, out2);
    RGS_CUDA(cudaGetLastError());
    ctx->launches += 2;
}
